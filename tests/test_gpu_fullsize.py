"""Full-size workloads, checked with what the oracle can afford at any size:
the whole result's canonical-order and threshold properties, and seeded
samples of supports (direct scans), downward closure and completeness.  The
planted workload is also compared bit-exactly with the full oracle run."""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen
from tests.fimcheck import check_canonical_arrays, sampled_checks

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
fim = pytest.importorskip("paper_2412_19420_gb300.fim")


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


def test_quest_10M_5000_sampled():
    c = datagen.quest_stress()
    ctx = fim.fim_create(0)
    try:
        got = _mine(ctx, c, 5000)
        st = fim.fim_get_stats(ctx)
    finally:
        fim.fim_destroy(ctx)
    assert st["pair_path"] == 1
    check_canonical_arrays(got.offsets, got.items, got.supports, 5000)
    sampled_checks(c, 5000, got.offsets, got.items, got.supports, k=150, ext=6)
    # singletons: every item's support, frequent or not, against a direct count
    sup = np.bincount(c.indices, minlength=c.m)
    single = {int(got.items[got.offsets[q]]): int(got.supports[q])
              for q in range(len(got)) if got.offsets[q + 1] - got.offsets[q] == 1}
    assert single == {j: int(s) for j, s in enumerate(sup) if s >= 5000}


def test_batched_4096_sampled(ctx):
    specs = datagen.batched_specs(4096)
    dbs = datagen.batched_dbs(specs)
    ms = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    fim.fim_mine_batched(ctx, dbs, ms)
    rng = np.random.default_rng(1)
    for d in rng.choice(len(dbs), 40, replace=False):
        got = fim.fim_fetch_batched(ctx, int(d))
        want = oracle.apriori(dbs[d].indptr, dbs[d].indices, dbs[d].m, ms[d])
        assert got.sha256() == want.sha256(), int(d)
