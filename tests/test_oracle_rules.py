"""Pins for the association-rule oracle (oracle/rules.py), independent of it.

The expected rules come from the definitions of confidence and lift applied
to supports recounted from the transactions (exact fractions, correctly
rounded once), and from closed forms: a database holding every subset of m
items once (independent items: conf = 2^-|Y|, lift = 1), an all-ones database
(conf = lift = 1, 3^m - 2^(m+1) + 1 rules) and disjoint co-occurring blocks
(conf = 1, lift = n / f).  The planted-mistake tests show that these pins
catch a swapped antecedent, a dropped n, a mirrored mask, a strict threshold
and a wrong consequent support.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import rules as orules
from paper_2412_19420_gb300 import datagen
from tests.fimcheck import bruteforce, dense


def _mine(c, thr):
    return oracle.apriori(c.indptr, c.indices, c.m, thr)


def _as_list(r):
    return [(int(q), int(m), float(cf), float(lf))
            for q, m, cf, lf in zip(r.set_index, r.ante_mask, r.conf, r.lift)]


def _bruteforce_rules(c, thr, ppm, max_len=20):
    """Rules from the definitions: supports counted on the dense matrix."""
    a = dense(c.indptr, c.indices, c.m)
    n = a.shape[0]

    def count(xs):
        return int(a[:, list(xs)].all(axis=1).sum()) if xs else n

    freq = bruteforce(c.indptr, c.indices, c.m, thr)
    order = sorted(freq, key=lambda x: (len(x), x))
    out = []
    for q, z in enumerate(order):
        if not 2 <= len(z) <= max_len:
            continue
        s_z = count(z)
        for mask in range(1, (1 << len(z)) - 1):
            x = tuple(v for i, v in enumerate(z) if mask >> i & 1)
            y = tuple(v for i, v in enumerate(z) if not mask >> i & 1)
            conf = Fraction(s_z, count(x))
            if conf >= Fraction(ppm, 10**6):
                out.append((q, mask, float(conf), float(conf / Fraction(count(y), n))))
    return out


# ---- brute force -----------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_bruteforce_random(seed):
    rng = np.random.default_rng(500 + seed)
    m = int(rng.integers(3, 10))
    n = int(rng.integers(5, 150))
    c = datagen.random_dense(n, m, float(rng.uniform(0.2, 0.8)), [seed, 11])
    thr = int(rng.integers(1, max(2, n // 5)))
    its = _mine(c, thr)
    for ppm in (0, 1, 250_000, 500_000, 800_000, 1_000_000):
        assert _as_list(orules.rules(its, n, ppm)) == _bruteforce_rules(c, thr, ppm)


def test_bruteforce_duplicates_and_empty_rows():
    rows = [[1, 1, 2], [], [2, 1, 0, 2], [3], [0, 1, 2, 3, 3, 3], [], [1, 2], [0, 2]]
    c = datagen.from_lists(rows, 4)
    its = _mine(c, 1)
    for ppm in (0, 400_000, 1_000_000):
        assert _as_list(orules.rules(its, len(rows), ppm)) == _bruteforce_rules(c, 1, ppm)


def test_max_len():
    c = datagen.random_dense(90, 8, 0.6, 3)
    its = _mine(c, 4)
    for ml in (2, 3, 5):
        got = _as_list(orules.rules(its, 90, 300_000, max_len=ml))
        assert got == _bruteforce_rules(c, 4, 300_000, max_len=ml)
    with pytest.raises(ValueError):
        orules.rules(its, 90, 300_000, max_len=1)
    with pytest.raises(ValueError):
        orules.rules(its, 90, 1_000_001)


# ---- closed forms ----------------------------------------------------------

def _binary_design(m):
    return datagen.from_lists([[j for j in range(m) if i >> j & 1] for i in range(1 << m)], m)


@pytest.mark.parametrize("ppm", [0, 125_000, 250_000, 500_000, 1_000_000])
def test_closed_form_independent_items(ppm):
    # every subset once: S(X) = 2^(m-|X|), so conf(X -> Y) = 2^-|Y| and lift = 1
    m = 7
    c = _binary_design(m)
    its = _mine(c, 1)
    r = orules.rules(its, 1 << m, ppm)
    off = its.offsets
    for q, mask, cf, lf in _as_list(r):
        L = int(off[q + 1] - off[q])
        ny = L - bin(mask).count("1")
        assert cf == 2.0 ** -ny and lf == 1.0
    want = sum(math.comb(m, L) * sum(math.comb(L, k) for k in range(1, L) if Fraction(1, 2**k) >= Fraction(ppm, 10**6))
               for L in range(2, m + 1))
    assert len(r) == want


def test_closed_form_all_ones():
    # every set has support n: conf = lift = 1; every ordered pair of disjoint
    # nonempty sets is a rule, 3^m - 2^(m+1) + 1 of them
    m, n = 7, 13
    c = datagen.from_lists([list(range(m))] * n, m)
    r = orules.rules(_mine(c, n), n, 1_000_000)
    assert len(r) == 3**m - 2 ** (m + 1) + 1
    assert set(r.conf.tolist()) == {1.0} and set(r.lift.tolist()) == {1.0}


def test_closed_form_disjoint_blocks():
    # block r (b_r items) fills f_r transactions of its own: rules only inside
    # a block, conf = 1 and lift = n / f_r
    blocks = [(range(0, 4), 30), (range(4, 9), 12), (range(9, 11), 5)]
    rows = []
    for items, f in blocks:
        rows += [list(items)] * f
    n = len(rows)
    c = datagen.from_lists(rows, 11)
    its = _mine(c, 1)
    r = orules.rules(its, n, 900_000)
    assert len(r) == sum(3 ** len(b) - 2 ** (len(b) + 1) + 1 for b, _ in blocks)
    assert set(r.conf.tolist()) == {1.0}
    off, items = its.offsets, its.items
    for q, _, _, lf in _as_list(r):
        first = int(items[off[q]])
        f = next(f for b, f in blocks if first in b)
        assert lf == n / f


def test_empty_and_singletons_only():
    c = datagen.from_lists([[i] for i in range(6)], 6)
    assert len(orules.rules(_mine(c, 1), 6, 0)) == 0
    c = datagen.from_lists([[]] * 4, 3)
    assert len(orules.rules(_mine(c, 1), 4, 0)) == 0


# ---- the pins catch planted mistakes --------------------------------------

def _pins_pass(mutant):
    for seed in range(4):
        rng = np.random.default_rng(900 + seed)
        m, n = int(rng.integers(4, 8)), int(rng.integers(20, 80))
        c = datagen.random_dense(n, m, 0.5, seed)
        its = _mine(c, 2)
        for ppm in (0, 500_000):
            if _as_list(orules.rules(its, n, ppm, _mutant=mutant)) != _bruteforce_rules(c, 2, ppm):
                return False
    # independent items at conf >= 1/2: exactly the rules with |Y| = 1
    c = _binary_design(5)
    if len(orules.rules(_mine(c, 1), 32, 500_000, _mutant=mutant)) != \
            sum(math.comb(5, L) * L for L in range(2, 6)):
        return False
    return True


def test_pins_pass_on_the_oracle():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(mutant):
    assert not _pins_pass(mutant)


# ---- stored output (tests/golden/oracle_hashes.json, written by make_golden.py)

def test_stored_rules_of_the_10k_x_169_workload():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_hashes.json")) as f:
        g = json.load(f)["grocery_like_10k_169"]
    c = datagen.grocery_like()
    assert c.sha256() == g["input_sha256"]
    its = _mine(c, g["minsup"])
    r = orules.rules(its, c.n, g["rules_min_conf_ppm"])
    assert len(r) == g["n_rules"] and r.sha256() == g["rules_sha256"]
