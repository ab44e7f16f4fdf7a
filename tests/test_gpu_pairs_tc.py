"""The tensor-core pair pass (tcgen05 kind::f8f6f4, f32 accumulator drained to
int32) against the oracle and the CUDA-core pair pass: bit-exact pair supports
for every tile shape at the edges, every drain length and every grid size."""
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


def _pairs(ctx, c, minsup, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags | fim.FIM_MAXLEN(2))
    return fim.fim_fetch_results(ctx), fim.fim_get_stats(ctx)


def test_tensor_core_path_is_taken(ctx):
    c = datagen.zipf_baskets(20_000, 300, 0.9, 8.0, 1)
    _, st = _pairs(ctx, c, 20)
    assert st["pair_path"] == 1


@pytest.mark.parametrize("n,m,seed", [(1000, 129, 1), (65_536, 255, 2), (300_001, 300, 3),
                                      (1_000_000, 140, 4)])
def test_tc_pairs_vs_oracle(ctx, n, m, seed):
    # tile edges (128, 129, 255, 256 items), ragged transaction tails, several K slices
    c = datagen.zipf_baskets(n, m, 0.7, 9.0, seed)
    minsup = max(1, n // 2000)
    got, st = _pairs(ctx, c, minsup)
    assert st["pair_path"] == 1
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup, max_len=2)
    assert got.sha256() == want.sha256()


@pytest.mark.parametrize("kdrain", [1, 7, 1024, 32768])
def test_tc_exact_on_all_ones(ctx, kdrain):
    # every pair support equals n: the largest partial sums the accumulator sees
    n, m = 262_145, 130
    indptr = np.arange(0, (n + 1) * m, m, dtype=np.int64)
    indices = np.tile(np.arange(m, dtype=np.int32), n)
    fim.fim_set_tuning(ctx, "pairs_kdrain", kdrain)
    try:
        fim.fim_build_bitmaps(ctx, indptr, indices, m)
        fim.fim_mine(ctx, n, fim.FIM_MAXLEN(2))
        got = fim.fim_fetch_results(ctx)
        assert fim.fim_get_stats(ctx)["pair_path"] == 1
    finally:
        fim.fim_set_tuning(ctx, "pairs_kdrain", 0)
    assert len(got) == m + m * (m - 1) // 2
    assert np.all(got.supports == n)


def test_tc_exact_at_the_f32_limit(ctx):
    # one CTA, one accumulator over 32,768 stages = 2^22 transactions of all
    # ones: the partial sum is 4 x 2^22 = 2^24, the largest integer an f32 run
    # holds exactly; one more transaction lands in a second segment
    n, m = (1 << 22) + 1, 3
    indptr = np.arange(0, (n + 1) * m, m, dtype=np.int64)
    indices = np.tile(np.arange(m, dtype=np.int32), n)
    fim.fim_set_tuning(ctx, "pairs_split", 1)
    fim.fim_set_tuning(ctx, "pairs_kdrain", 32768)
    try:
        fim.fim_build_bitmaps(ctx, indptr, indices, m)
        fim.fim_mine(ctx, n, fim.FIM_MAXLEN(2))
        got = fim.fim_fetch_results(ctx)
        assert fim.fim_get_stats(ctx)["pair_path"] == 1
    finally:
        fim.fim_set_tuning(ctx, "pairs_split", 0)
        fim.fim_set_tuning(ctx, "pairs_kdrain", 0)
    assert len(got) == m + m * (m - 1) // 2
    assert np.all(got.supports == n)


@pytest.mark.parametrize("split", [1, 3, 17, 1000])
def test_tc_split_k_invariant(ctx, split):
    c = datagen.zipf_baskets(200_000, 260, 0.8, 7.0, 9)
    fim.fim_set_tuning(ctx, "pairs_split", split)
    try:
        got, _ = _pairs(ctx, c, 100)
    finally:
        fim.fim_set_tuning(ctx, "pairs_split", 0)
    ref, st = _pairs(ctx, c, 100, fim.FIM_PAIRS_POPC)
    assert st["pair_path"] == 0
    assert got.sha256() == ref.sha256()


def test_tuning_keys_validated(ctx):
    with pytest.raises(fim.FimError):
        fim.fim_set_tuning(ctx, "pairs_kdrain", 40000)
    with pytest.raises(fim.FimError):
        fim.fim_set_tuning(ctx, "no_such_knob", 1)
