"""Class representations (dense bitmap / diffset) and DFS traces.

The representation a class is counted in must never change a support: every
mode is compared bit-exactly with the oracle.  Traces are checked against
invariants that hold for any correct accounting.
"""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _mine(ctx, c, minsup, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags)
    return fim.fim_fetch_results(ctx), fim.fim_get_stats(ctx)


CASES = [
    ("planted", lambda: datagen.planted(n=20_000, m=800, n_patterns=60, seed=4), 100),
    ("zipf", lambda: datagen.zipf_baskets(30_000, 300, 1.0, 9.0, 21), 60),
    ("dense", lambda: datagen.random_dense(3000, 14, 0.6, 5), 200),
]


@pytest.mark.parametrize("name,gen,minsup", CASES, ids=[c[0] for c in CASES])
def test_diffset_rule_is_exact(ctx, name, gen, minsup):
    c = gen()
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup)
    got, st = _mine(ctx, c, minsup, fim.FIM_DIFFSET_RULE)
    assert got.sha256() == want.sha256()
    if name in ("planted", "dense"):
        assert st["diffset_classes"] > 0


def test_touched_bytes_bounded_by_dense_bytes(ctx):
    # FIM_NO_SPLIT keeps every subtree in its worker, so the byte counts do not
    # depend on how the run happened to split work
    c = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    _, plain = _mine(ctx, c, 100, fim.FIM_NO_SPLIT)
    _, rule = _mine(ctx, c, 100, fim.FIM_NO_SPLIT | fim.FIM_DIFFSET_RULE)
    assert 0 < plain["dfs_touched_bytes"] <= plain["dfs_bytes"]
    assert rule["dfs_words"] == plain["dfs_words"]            # same classes, same candidates
    assert rule["dfs_bytes"] == plain["dfs_bytes"]
    assert rule["dfs_touched_bytes"] < plain["dfs_touched_bytes"]  # diffsets skip more sectors


def _traces(ctx):
    return fim.fim_fetch_traces(ctx)


def test_traces_account_for_every_class(ctx):
    c = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    got, st = _mine(ctx, c, 100, fim.FIM_TRACE)
    want = oracle.apriori(c.indptr, c.indices, c.m, 100)
    assert got.sha256() == want.sha256()          # tracing never changes results
    X, Y = _traces(ctx)
    assert len(X) == st["classes"]                # one row per class pass
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(Y))
    assert set(np.unique(Y[:, 1])) <= {0.0, 1.0}
    # the root classes' subtrees partition all the DFS work (feature 0 = |Y|/16)
    roots = X[:, 0] == np.float32(2 / 16)
    total = np.sum(np.exp2(Y[roots, 0].astype(np.float64)) - 1.0)
    assert total == pytest.approx(st["dfs_words"], rel=1e-5)
    # a class's subtree work is at least its own candidate words (feature 3 = log2(1+k)/16)
    own = (np.exp2(16.0 * X[:, 3].astype(np.float64)) - 1.0) * ((c.n + 31) // 32)
    assert np.all(np.exp2(Y[:, 0].astype(np.float64)) - 1.0 >= own * (1 - 1e-5))


def test_trace_requires_trace_flag(ctx):
    c = datagen.zipf_baskets(2000, 30, 0.9, 5.0, 3)
    _mine(ctx, c, 20)
    with pytest.raises(fim.FimError) as e:
        _traces(ctx)
    assert e.value.code == fim.FIM_E_STATE


def test_learned_mode_needs_weights(ctx):
    c2 = fim.fim_create(0)
    try:
        c = datagen.zipf_baskets(2000, 30, 0.9, 5.0, 3)
        fim.fim_build_bitmaps(c2, c.indptr, c.indices, c.m)
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine(c2, 20, fim.FIM_LEARNED)
        assert e.value.code == fim.FIM_E_STATE
    finally:
        fim.fim_destroy(c2)


@pytest.mark.parametrize("seed", [0, 1])
def test_learned_mode_is_exact_with_any_weights(ctx, seed):
    # even untrained (random) weights may only change order and representation
    w = datagen.mlp_init_weights(seed)
    w[-1] = 5.0 if seed else -5.0   # push the diffset logit to both extremes
    fim.fim_sched_load_weights(ctx, w)
    for _, gen, minsup in CASES:
        c = gen()
        got, _ = _mine(ctx, c, minsup, fim.FIM_LEARNED)
        want = oracle.apriori(c.indptr, c.indices, c.m, minsup)
        assert got.sha256() == want.sha256()
