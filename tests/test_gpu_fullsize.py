"""Full-size workloads, compared bit for bit with the oracle's whole answer.

The oracle's canonical result for the 10^7 x 5,000 workload and for every
database of the 4,096-database batch is recorded in
tests/golden/oracle_hashes.json by tests/golden/make_golden.py, which calls
only the oracle; the tests use it when their regenerated input has the
recorded sha256, and run the oracle live otherwise.  The canonical-order and
threshold properties are checked on the GPU's output as well.  The planted
workload is compared with a live oracle run.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen
from tests.fimcheck import check_canonical_arrays

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
fim = pytest.importorskip("paper_2412_19420_gb300.fim")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_hashes.json")


def _golden(name):
    with open(GOLDEN) as f:
        return json.load(f).get(name)


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _mine(ctx, c, minsup, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags)
    return fim.fim_fetch_results(ctx)


def test_planted_100k_2000_full_oracle(ctx):
    c = datagen.planted(seed=0)
    got = _mine(ctx, c, 500)
    want = oracle.apriori(c.indptr, c.indices, c.m, 500)
    assert got.sha256() == want.sha256()
    rule = _mine(ctx, c, 500, fim.FIM_DIFFSET_RULE)
    assert rule.sha256() == want.sha256()


def test_quest_10M_5000_full():
    c = datagen.quest_stress()
    ctx = fim.fim_create(0)
    try:
        got = _mine(ctx, c, 5000)
        st = fim.fim_get_stats(ctx)
    finally:
        fim.fim_destroy(ctx)
    assert st["pair_path"] == 1
    check_canonical_arrays(got.offsets, got.items, got.supports, 5000)
    g = _golden("quest_10M_5000")
    if g is not None and g["input_sha256"] == c.sha256() and g["minsup"] == 5000:
        assert len(got) == g["n_sets"]
        assert got.sha256() == g["result_sha256"]
    else:
        want = oracle.apriori(c.indptr, c.indices, c.m, 5000)
        assert got.sha256() == want.sha256()


def _batch_digests(dbs, ms, result_hashes):
    """sha256 over the databases' input sha256 and threshold, and over their
    result sha256, in database order (the recorded batch digests)."""
    hi, hr = hashlib.sha256(), hashlib.sha256()
    for c, m, r in zip(dbs, ms, result_hashes):
        hi.update(f"{c.sha256()}:{int(m)};".encode())
        hr.update(r.encode())
    return hi.hexdigest(), hr.hexdigest()


def _slice(res, s0, s1):
    o = res.offsets[s0:s1 + 1].astype(np.uint64)
    return fim.Itemsets(o - o[0], res.items[int(o[0]):int(o[-1])], res.supports[s0:s1])


@pytest.mark.parametrize("flags", [0, "learned"])
def test_batched_4096_full(ctx, flags):
    dbs = datagen.batched_dbs(datagen.batched_specs(4096))
    ms = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    if flags == "learned":
        # any weights give exact counts; seeded starting weights steer here
        fim.fim_sched_load_weights(ctx, datagen.mlp_init_weights(3))
        flags = fim.FIM_LEARNED
    fim.fim_mine_batched(ctx, dbs, ms, flags=flags)
    res = fim.fim_fetch_batched(ctx, fim.FIM_ALL_DBS)
    sl = fim.fim_batch_slices(ctx, len(dbs)).astype(np.int64)
    assert sl[0] == 0 and sl[-1] == len(res) and (np.diff(sl) >= 0).all()
    got = []
    for d in range(len(dbs)):
        part = _slice(res, sl[d], sl[d + 1])
        check_canonical_arrays(part.offsets, part.items, part.supports, ms[d])
        got.append(part.sha256())
    g = _golden("batched_4096")
    di, dr = _batch_digests(dbs, ms, got)
    if g is not None and g["input_sha256"] == di:
        assert len(res) == g["n_sets"]
        if dr != g["result_sha256"]:  # name the first database that differs
            for d in range(len(dbs)):
                want = oracle.apriori(dbs[d].indptr, dbs[d].indices, dbs[d].m, ms[d])
                assert got[d] == want.sha256(), d
        assert dr == g["result_sha256"]
    else:
        for d in range(len(dbs)):
            want = oracle.apriori(dbs[d].indptr, dbs[d].indices, dbs[d].m, ms[d])
            assert got[d] == want.sha256(), d
