"""Pins for the CPU oracle (oracle/apriori.c), independent of the oracle's code.

Each check is fixed by the mathematics of Eq. 1-3 rather than by the oracle:
brute-force enumeration, closed-form databases, numpy column sums and A^T A,
and invariants.  The planted-mistake tests build copies of the oracle with one
deliberate error and show that these pins catch each of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen
from tests.fimcheck import bruteforce, check_invariants, dense


def _ap(c, thr, **kw):
    return oracle.apriori(c.indptr, c.indices, c.m, thr, **kw)


# ---- brute force on tiny random databases (all 2^m - 1 subsets) ----------

@pytest.mark.parametrize("density", [0.0, 0.05, 0.3, 0.7, 1.0])
@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_random(density, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(3, 11))
    n = int(rng.integers(1, 120))
    c = datagen.random_dense(n, m, density, [seed, 7])
    for thr in sorted({1, 2, max(1, n // 10), max(1, n // 3), n}):
        for strict in (False, True):
            got = _ap(c, thr, strict=strict, threads=3).as_dict()
            assert got == bruteforce(c.indptr, c.indices, m, thr, strict)


def test_bruteforce_with_duplicates_and_empty_rows():
    # duplicates inside a transaction collapse (Eq. 1 is set membership);
    # empty transactions count toward n and contain nothing
    rows = [[1, 1, 2], [], [2, 1, 0, 2], [3], [0, 1, 2, 3, 3, 3], [], [1, 2]]
    c = datagen.from_lists(rows, 4)
    for thr in (1, 2, 3):
        assert _ap(c, thr).as_dict() == bruteforce(c.indptr, c.indices, 4, thr)


def test_bruteforce_many_seeds_mid_density():
    for seed in range(40):
        rng = np.random.default_rng(1000 + seed)
        m = int(rng.integers(8, 13))
        n = int(rng.integers(20, 256))
        c = datagen.random_dense(n, m, float(rng.uniform(0.2, 0.6)), seed)
        thr = int(rng.integers(1, max(2, n // 4)))
        assert _ap(c, thr, threads=2).as_dict() == bruteforce(c.indptr, c.indices, m, thr)


# ---- closed forms ----------------------------------------------------------

def _binary_design(m):
    n = 1 << m
    return datagen.from_lists([[j for j in range(m) if i >> j & 1] for i in range(n)], m)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 10])
def test_closed_form_binary_design(k):
    # T_i = {j : bit j of i}, n = 2^m: S(X) = 2^(m-|X|); at minsup 2^(m-k)
    # exactly the sets of size <= k are frequent: sum_{j<=k} C(m, j) of them
    m = 10
    c = _binary_design(m)
    got = _ap(c, 1 << (m - k)).as_dict()
    assert len(got) == sum(math.comb(m, j) for j in range(1, k + 1))
    assert all(s == 1 << (m - len(x)) for x, s in got.items())
    # strict at the same threshold keeps only the sizes < k
    got_s = _ap(c, 1 << (m - k), strict=True).as_dict()
    assert len(got_s) == sum(math.comb(m, j) for j in range(1, k))


def test_closed_form_all_ones():
    m, n = 12, 37
    c = datagen.from_lists([list(range(m))] * n, m)
    got = _ap(c, n).as_dict()
    assert len(got) == (1 << m) - 1 and set(got.values()) == {n}
    assert _ap(c, n + 1).as_dict() == {}


def test_closed_form_identity():
    m = 50
    c = datagen.from_lists([[i] for i in range(m)], m)
    got = _ap(c, 1).as_dict()
    assert got == {(i,): 1 for i in range(m)}
    assert _ap(c, 2).as_dict() == {}


def test_closed_form_disjoint_blocks():
    # block r (items B_r, |B_r| = b_r) fills f_r transactions of its own:
    # F is the union of the power sets of the blocks with f_r >= minsup
    blocks = [(range(0, 4), 30), (range(4, 9), 12), (range(9, 11), 5), (range(11, 17), 20)]
    rows = []
    for items, f in blocks:
        rows += [list(items)] * f
    c = datagen.from_lists(rows, 17)
    for thr in (5, 12, 20, 31):
        want = {}
        for items, f in blocks:
            if f >= thr:
                for k in range(1, len(items) + 1):
                    for x in itertools.combinations(items, k):
                        want[x] = f
        assert _ap(c, thr).as_dict() == want


def test_minsup_from_ppm():
    assert datagen.minsup_from_ppm(10_000, 10_000) == 100
    assert datagen.minsup_from_ppm(1_000_000, 1_000) == 1000
    assert datagen.minsup_from_ppm(12_345, 20_000) == 247  # ceil(246.9)
    assert datagen.minsup_from_ppm(10, 1) == 1


# ---- library cross-checks: column sums and A^T A ------------------------

def test_singletons_and_pairs_match_numpy():
    c = datagen.grocery_like()
    a = dense(c.indptr, c.indices, c.m).astype(np.int64)
    col = a.sum(0)
    gram = a.T @ a
    thr = 100
    got = _ap(c, thr, max_len=2).as_dict()
    want = {(j,): int(col[j]) for j in range(c.m) if col[j] >= thr}
    for i in range(c.m):
        for j in range(i + 1, c.m):
            if gram[i, j] >= thr and col[i] >= thr and col[j] >= thr:
                want[(i, j)] = int(gram[i, j])
    assert got == want


def test_item_supports_sum_to_nnz():
    c = datagen.grocery_like(seed=3)
    got = _ap(c, 1, max_len=1)
    assert int(got.supports.sum()) == c.nnz  # generator rows are distinct


def test_support_many_matches_dense():
    c = datagen.random_dense(300, 12, 0.4, 5)
    a = dense(c.indptr, c.indices, c.m)
    rng = np.random.default_rng(0)
    qs = [tuple(sorted(rng.choice(12, size=int(rng.integers(1, 6)), replace=False)))
          for _ in range(50)]
    got = oracle.support_many(c.indptr, c.indices, c.m, qs, threads=3)
    want = [int(a[:, list(q)].all(1).sum()) for q in qs]
    assert got.tolist() == want


# ---- invariants and determinism on a realistic workload ------------------

def test_invariants_grocery_like():
    c = datagen.grocery_like()
    r = _ap(c, 100)
    d = r.as_dict()
    item_sup = np.bincount(c.indices, minlength=c.m)
    order = [tuple(int(v) for v in r.items[r.offsets[q]:r.offsets[q + 1]]) for q in range(len(r))]
    check_invariants(d, 100, item_support=item_sup, order=order)
    # completeness one level up: no frequent extension of a frequent set is missing
    a = dense(c.indptr, c.indices, c.m)
    for x in d:
        rows = a[:, list(x)].all(1)
        ext = (a[rows] .sum(0))
        for j in range(max(x) + 1, c.m):
            if ext[j] >= 100:
                assert x + (j,) in d


def test_thread_count_does_not_change_result():
    c = datagen.zipf_baskets(3000, 60, 0.9, 7.0, 11)
    h = {_ap(c, 30, threads=t).sha256() for t in (1, 2, 5, 8)}
    assert len(h) == 1


def test_strict_equals_next_threshold():
    c = datagen.zipf_baskets(2000, 40, 0.8, 6.0, 4)
    for thr in (10, 25, 60):
        assert _ap(c, thr, strict=True).sha256() == _ap(c, thr + 1).sha256()


def test_malformed_input_rejected():
    with pytest.raises(ValueError):
        oracle.apriori(np.array([0, 2, 1]), np.array([0, 1], np.int32), 3, 1)
    with pytest.raises(ValueError):
        oracle.apriori(np.array([0, 2]), np.array([0, 5], np.int32), 3, 1)


def test_empty_database():
    c = datagen.from_lists([], 5)
    assert len(_ap(c, 1)) == 0
    c = datagen.from_lists([[], [], []], 5)
    assert len(_ap(c, 1)) == 0


# ---- planted mistakes: each must fail at least one pin -------------------

def _pins_pass(mutant: int) -> bool:
    try:
        for seed in range(4):
            c = datagen.random_dense(64, 8, 0.45, [seed, 99])
            for thr in (1, 9, 17):
                if oracle.apriori(c.indptr, c.indices, c.m, thr, _mutant=mutant).as_dict() \
                        != bruteforce(c.indptr, c.indices, c.m, thr):
                    return False
        rows = [[1, 1, 2], [2, 1, 0, 2], [0, 1, 2, 3, 3]]
        c = datagen.from_lists(rows, 4)
        if oracle.apriori(c.indptr, c.indices, 4, 1, _mutant=mutant).as_dict() \
                != bruteforce(c.indptr, c.indices, 4, 1):
            return False
        c = _binary_design(8)
        got = oracle.apriori(c.indptr, c.indices, 8, 1 << 5, _mutant=mutant).as_dict()
        if len(got) != sum(math.comb(8, j) for j in range(1, 4)):
            return False
    except (ValueError, MemoryError):
        return False
    return True


def test_pins_pass_on_the_oracle():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(mutant):
    assert not _pins_pass(mutant)
