"""Test helpers shared by the oracle and GPU tests (no mining code here).

* ``bruteforce``: every non-empty subset of the items, supports counted on a
  dense 0/1 matrix -- the definition of Eq. 1-3 written out for tiny inputs.
* ``check_invariants``: properties any correct answer has (downward closure,
  anti-monotone supports, threshold, canonical order, no duplicates).
"""
from __future__ import annotations

import itertools

import numpy as np


def dense(indptr, indices, m) -> np.ndarray:
    n = len(indptr) - 1
    a = np.zeros((n, m), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    a[rows, np.asarray(indices, dtype=np.int64)] = True
    return a


def bruteforce(indptr, indices, m, threshold, strict=False) -> dict:
    """{itemset tuple: support} over all 2^m - 1 subsets (m <= 16)."""
    assert m <= 16
    a = dense(indptr, indices, m)
    rowmask = (a.astype(np.int64) << np.arange(m, dtype=np.int64)).sum(1)
    out = {}
    masks = np.arange(1, 1 << m, dtype=np.int64)
    sup = ((rowmask[:, None] & masks[None, :]) == masks[None, :]).sum(0)
    for mask, s in zip(masks.tolist(), sup.tolist()):
        if (s > threshold) if strict else (s >= threshold):
            out[tuple(j for j in range(m) if mask >> j & 1)] = int(s)
    return out


def canonical_order_ok(sets: list[tuple]) -> bool:
    keys = [(len(x), x) for x in sets]
    return all(keys[i] < keys[i + 1] for i in range(len(keys) - 1)) and \
        all(list(x) == sorted(set(x)) for x in sets)


def check_canonical_arrays(offsets, items, supports, threshold):
    """Whole-result checks on the canonical arrays (any size): items strictly
    ascending inside each set, sets ordered by (size, lexicographic) with no
    duplicates, every support >= threshold."""
    offsets = np.asarray(offsets, np.int64)
    items = np.asarray(items, np.int64)
    lens = np.diff(offsets)
    assert np.all(lens >= 1)
    assert np.all(np.diff(lens) >= 0), "sets not ordered by size"
    assert np.all(np.asarray(supports, np.int64) >= threshold)
    for L in np.unique(lens):
        sel = np.nonzero(lens == L)[0]
        rows = items[offsets[sel][:, None] + np.arange(L)[None, :]]
        if L > 1:
            assert np.all(np.diff(rows, axis=1) > 0), "items not ascending inside a set"
        if len(rows) > 1:
            diff = rows[1:] != rows[:-1]
            assert np.all(diff.any(1)), "duplicate set"
            first = diff.argmax(1)
            r = np.arange(len(first))
            assert np.all(rows[1:][r, first] > rows[:-1][r, first]), "sets not lexicographic"


def sampled_checks(csr, threshold, offsets, items, supports, k=200, ext=8, seed=0):
    """Checks the oracle can afford at any size, on a seeded sample:
    supports of sampled sets by a direct scan, their (|X|-1)-subsets reported
    with supports >= theirs, and completeness one level up (a sampled
    extension X u {e} is reported iff its scanned support reaches threshold)."""
    import oracle
    offsets = np.asarray(offsets, np.int64)
    items = np.asarray(items, np.int64)
    R = len(supports)
    if R == 0:
        return
    keyset = {}
    for q in range(R):
        keyset[items[offsets[q]:offsets[q + 1]].tobytes()] = int(supports[q])
    rng = np.random.default_rng(seed)
    pick = rng.choice(R, size=min(k, R), replace=False)
    sets = [tuple(items[offsets[q]:offsets[q + 1]]) for q in pick]
    scanned = oracle.support_many(csr.indptr, csr.indices, csr.m, sets)
    for q, x, s in zip(pick, sets, scanned):
        assert int(s) == int(supports[q]), (x, int(s), int(supports[q]))
        if len(x) > 1:
            for sub in itertools.combinations(x, len(x) - 1):
                key = np.asarray(sub, np.int64).tobytes()
                assert key in keyset, ("missing subset", sub)
                assert keyset[key] >= int(s)
    queries = []
    for x in sets:
        for e in rng.choice(csr.m, size=min(ext, csr.m), replace=False):
            if e not in x:
                queries.append(tuple(sorted(x + (int(e),))))
    scanned = oracle.support_many(csr.indptr, csr.indices, csr.m, queries)
    for y, s in zip(queries, scanned):
        reported = np.asarray(y, np.int64).tobytes() in keyset
        assert reported == (int(s) >= threshold), ("completeness", y, int(s))


def check_invariants(result: dict, threshold: int, strict=False, item_support=None,
                     order: list | None = None) -> None:
    """Raise AssertionError unless ``result`` ({set: support}) is consistent."""
    for x, s in result.items():
        assert (s > threshold) if strict else (s >= threshold), (x, s)
        assert len(x) == len(set(x)) and list(x) == sorted(x), x
        if len(x) > 1:
            for sub in itertools.combinations(x, len(x) - 1):
                assert sub in result, ("downward closure", x, sub)
                assert result[sub] >= s, ("anti-monotone", x, sub)
        elif item_support is not None:
            assert item_support[x[0]] == s, ("singleton", x)
    if item_support is not None:
        for j, s in enumerate(item_support):
            if (s > threshold) if strict else (s >= threshold):
                assert (j,) in result, ("missing frequent item", j)
    if order is not None:
        assert canonical_order_ok(order)
