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
