"""Failure detection without a GPU fault: a bounded device wait that runs out.

The DFS work queue's waits (a worker waiting for a pushed task to be
published, workers waiting for the queue to drain) spin against a
%globaltimer limit.  The test withholds one publish through the
"test_withhold_task" hook and shortens the limit to 200 ms: the mine must end
with FIM_E_TIMEOUT within a few seconds, and the same ctx must then mine
correctly.  Nothing traps, faults or hangs.
"""
import time

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


def _queue_case(ctx):
    """A workload whose mine pushes classes to the device queue."""
    for c, thr in [(datagen.planted(n=20_000, m=600, n_patterns=40, seed=9), 120),
                   (datagen.planted(n=20_000, m=800, n_patterns=60, seed=4), 100)]:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, thr)
        if fim.fim_get_stats(ctx)["tasks_pushed"] > 0:
            return c, thr
    pytest.fail("no workload pushed tasks to the queue")


def test_withheld_publish_times_out_and_ctx_survives(ctx):
    c, thr = _queue_case(ctx)
    want = oracle.apriori(c.indptr, c.indices, c.m, thr).sha256()
    fim.fim_set_tuning(ctx, "spin_limit_ms", 200)
    fim.fim_set_tuning(ctx, "test_withhold_task", 0)
    try:
        t0 = time.perf_counter()
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine(ctx, thr)
        elapsed = time.perf_counter() - t0
        assert e.value.args[0].endswith(f"({fim.FIM_E_TIMEOUT})")
        assert elapsed < 10.0
        with pytest.raises(fim.FimError):  # nothing is held after the failed mine
            fim.fim_fetch_results(ctx)
    finally:
        fim.fim_set_tuning(ctx, "test_withhold_task", -1)
        fim.fim_set_tuning(ctx, "spin_limit_ms", 60_000)
    fim.fim_mine(ctx, thr)  # the same ctx, the same matrix: exact again
    assert fim.fim_fetch_results(ctx).sha256() == want
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, thr)
    assert fim.fim_fetch_results(ctx).sha256() == want


def test_spin_limit_knob_range(ctx):
    for key, bad in (("spin_limit_ms", 0), ("spin_limit_ms", 600_001), ("test_withhold_task", -2)):
        with pytest.raises(fim.FimError):
            fim.fim_set_tuning(ctx, key, bad)


def test_debug_checks_pass_on_correct_runs(ctx):
    # guard words (pad bits and words of every column) after the build and the
    # canonical-output invariants after the mine, for ragged and degenerate sizes
    fim.fim_set_tuning(ctx, "debug_checks", 1)
    try:
        cases = [(datagen.zipf_baskets(70_001, 200, 0.9, 6.0, 3), 250, 0),
                 (datagen.zipf_baskets(4_096, 60, 0.9, 6.0, 4), 10, fim.FIM_STRICT),
                 (datagen.random_dense(33, 9, 0.6, 5), 3, fim.FIM_MAXLEN(3)),
                 (datagen.from_lists([[]] * 7, 4), 1, 0)]
        for c, thr, flags in cases:
            fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
            fim.fim_mine(ctx, thr, flags)
            want = oracle.apriori(c.indptr, c.indices, c.m, thr, strict=bool(flags & fim.FIM_STRICT),
                                  max_len=3 if flags == fim.FIM_MAXLEN(3) else 0)
            assert fim.fim_fetch_results(ctx).sha256() == want.sha256()
    finally:
        fim.fim_set_tuning(ctx, "debug_checks", 0)
