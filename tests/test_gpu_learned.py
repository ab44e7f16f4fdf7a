"""What the trained scheduling network gains over the miner without it.

The network is trained on the GPU (libfim's own kernels) from the plain
miner's traces of one planted database and judged on a held-out one:
  * results stay bit-exact (the network never changes a count);
  * its work and representation predictions beat the trivial predictors,
    scored against the plain miner's measured traces;
  * the learned miner streams fewer bytes than the plain miner (diffset
    classes skip the sectors a dense bitmap would read);
  * the root order from the network's work prediction is exact too.
"""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
sched = pytest.importorskip("paper_2412_19420_gb300.sched")


@pytest.fixture(scope="module")
def trained():
    ctx = fim.fim_create(0)
    train_db = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    x, t = sched.collect_traces(ctx, train_db, 100)
    w, hist = sched.fit(ctx, x, t, steps=1500, lr=2e-3, seed=0)
    yield ctx, w, hist
    fim.fim_destroy(ctx)


def _mine(ctx, c, minsup, flags):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags)
    return fim.fim_fetch_results(ctx), fim.fim_get_stats(ctx)


def test_training_converged(trained):
    _, _, hist = trained
    assert np.mean(hist[-50:]) < 0.25 * np.mean(hist[:10])


def test_predictions_beat_trivial_predictors_on_held_out_traces(trained):
    ctx, w, _ = trained
    held = datagen.planted(n=20_000, m=800, n_patterns=60, seed=5)
    x, t = sched.collect_traces(ctx, held, 100)
    ev = sched.evaluate(ctx, w, x, t)
    majority = max(np.mean(t[:, 1] > 0.5), 1 - np.mean(t[:, 1] > 0.5))
    assert ev["work_r2"] > 0.5, ev          # predicting the mean scores 0
    assert ev["repr_accuracy"] > majority, (ev, majority)


def test_learned_miner_is_exact_and_streams_fewer_bytes(trained):
    ctx, w, _ = trained
    fim.fim_sched_load_weights(ctx, w)
    held = datagen.planted(n=20_000, m=800, n_patterns=60, seed=5)
    want = oracle.apriori(held.indptr, held.indices, held.m, 100)
    plain, sp = _mine(ctx, held, 100, fim.FIM_NO_SPLIT)
    # every class consults the network (by default only classes with >= 8
    # candidates do, where the choice can pay for the inference)
    fim.fim_set_tuning(ctx, "learned_kmin", 1)
    try:
        learned, sl = _mine(ctx, held, 100, fim.FIM_LEARNED | fim.FIM_NO_SPLIT)
    finally:
        fim.fim_set_tuning(ctx, "learned_kmin", 8)
    rule, sr = _mine(ctx, held, 100, fim.FIM_DIFFSET_RULE | fim.FIM_NO_SPLIT)
    default, sd = _mine(ctx, held, 100, fim.FIM_LEARNED | fim.FIM_NO_SPLIT)
    assert default.sha256() == want.sha256()
    assert sd["dfs_touched_bytes"] <= sp["dfs_touched_bytes"]
    assert plain.sha256() == want.sha256()
    assert learned.sha256() == want.sha256()
    assert rule.sha256() == want.sha256()
    assert sl["diffset_classes"] > 0
    # the network's representation choice streams fewer bytes than the plain
    # miner, and about as few as the closed-form size rule
    assert sl["dfs_touched_bytes"] < 0.9 * sp["dfs_touched_bytes"], (sl, sp)
    assert sl["dfs_touched_bytes"] < 1.05 * sr["dfs_touched_bytes"], (sl, sr)


def test_learned_root_order_is_exact(trained):
    ctx, w, _ = trained
    fim.fim_sched_load_weights(ctx, w)
    held = datagen.planted(n=20_000, m=800, n_patterns=60, seed=5)
    want = oracle.apriori(held.indptr, held.indices, held.m, 100)
    fim.fim_set_tuning(ctx, "learned_order", 1)
    try:
        got, _ = _mine(ctx, held, 100, fim.FIM_LEARNED)
    finally:
        fim.fim_set_tuning(ctx, "learned_order", 0)
    assert got.sha256() == want.sha256()
