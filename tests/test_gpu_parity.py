"""GPU miner vs the CPU oracle: bit-exact canonical results (integer work).

Every test calls the CUDA path through the C ABI (paper_2412_19420_gb300.fim)
and compares the canonical byte stream (offsets, items, supports) with the
oracle's on the same seeded input.
"""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen
from tests.fimcheck import check_invariants

pytestmark = pytest.mark.gpu

fim = pytest.importorskip("paper_2412_19420_gb300.fim")


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _gpu(ctx, c, minsup, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags)
    return fim.fim_fetch_results(ctx)


def _same(ctx, c, minsup, flags=0, strict=False, max_len=0):
    got = _gpu(ctx, c, minsup, flags)
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup, strict=strict, max_len=max_len)
    if got.sha256() != want.sha256():
        g, w = got.as_dict(), want.as_dict()
        missing = [k for k in w if k not in g][:5]
        extra = [k for k in g if k not in w][:5]
        wrong = [(k, g[k], w[k]) for k in w if k in g and g[k] != w[k]][:5]
        raise AssertionError(f"{len(got)} vs {len(want)} sets; missing {missing} extra {extra} "
                             f"wrong {wrong}")
    return got


@pytest.mark.parametrize("density", [0.0, 0.05, 0.3, 0.7, 1.0])
@pytest.mark.parametrize("seed", range(3))
def test_random_dense_small(ctx, density, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(2, 14))
    c = datagen.random_dense(n, m, density, [seed, 3])
    for thr in sorted({1, 2, max(1, n // 7), n}):
        _same(ctx, c, thr)


def test_tiles_and_ragged_tails(ctx):
    # several word chunks, several 64-item pair tiles, ragged last word
    for n, m, s in [(33, 70, 1), (4097, 130, 2), (70_001, 200, 3), (12_345, 65, 4)]:
        c = datagen.zipf_baskets(n, m, 0.9, 6.0, s)
        _same(ctx, c, max(2, n // 200))


def test_duplicates_and_empty_transactions(ctx):
    rows = [[1, 1, 2], [], [2, 1, 0, 2], [3], [0, 1, 2, 3, 3, 3], [], [1, 2]] * 5
    c = datagen.from_lists(rows, 4)
    for thr in (1, 5, 10, 15, 35):
        _same(ctx, c, thr)


def test_all_ones_deep(ctx):
    # every subset frequent: 2^14 - 1 sets, the deepest DFS the lattice allows
    m = 14
    c = datagen.from_lists([list(range(m))] * 50, m)
    got = _same(ctx, c, 50)
    assert len(got) == (1 << m) - 1


def test_binary_design(ctx):
    m = 12
    c = datagen.from_lists([[j for j in range(m) if i >> j & 1] for i in range(1 << m)], m)
    for k in (1, 2, 4, 7):
        _same(ctx, c, 1 << (m - k))


def test_strict_threshold(ctx):
    c = datagen.zipf_baskets(3000, 50, 0.8, 6.0, 9)
    for thr in (0, 20, 60):
        got = _gpu(ctx, c, thr, fim.FIM_STRICT)
        want = oracle.apriori(c.indptr, c.indices, c.m, thr, strict=True)
        assert got.sha256() == want.sha256()


def test_max_len(ctx):
    c = datagen.zipf_baskets(5000, 60, 0.8, 8.0, 5)
    for L in (1, 2, 3):
        got = _gpu(ctx, c, 25, fim.FIM_MAXLEN(L))
        want = oracle.apriori(c.indptr, c.indices, c.m, 25, max_len=L)
        assert got.sha256() == want.sha256()


def test_grocery_like_full(ctx):
    c = datagen.grocery_like()
    _same(ctx, c, 100)


def test_no_split_equals_split(ctx):
    c = datagen.zipf_baskets(20_000, 300, 1.0, 9.0, 21)
    a = _gpu(ctx, c, 60).sha256()
    b = _gpu(ctx, c, 60, fim.FIM_NO_SPLIT).sha256()
    assert a == b


def test_pair_paths_agree(ctx):
    c = datagen.zipf_baskets(30_000, 400, 0.9, 7.0, 8)
    a = _gpu(ctx, c, 50).sha256()
    b = _gpu(ctx, c, 50, fim.FIM_PAIRS_POPC).sha256()
    assert a == b


def test_device_input_equals_host_input(ctx):
    import torch
    c = datagen.zipf_baskets(10_000, 150, 0.9, 6.0, 12)
    host = _gpu(ctx, c, 50)
    ip = torch.from_numpy(c.indptr).cuda()
    ix = torch.from_numpy(c.indices).cuda()
    fim.fim_build_bitmaps(ctx, ip, ix, c.m)
    fim.fim_mine(ctx, 50)
    dev = fim.fim_fetch_results(ctx)
    assert dev.sha256() == host.sha256()
    # device output buffers
    R, T = fim.fim_result_sizes(ctx)
    out = (torch.empty(R + 1, dtype=torch.int64, device="cuda"),
           torch.empty(T, dtype=torch.int32, device="cuda"),
           torch.empty(R, dtype=torch.int32, device="cuda"))
    fim.fim_fetch_results(ctx, out)
    assert np.array_equal(out[2].cpu().numpy().view(np.uint32), host.supports)


def test_errors_are_reported(ctx):
    c2 = fim.fim_create(0)
    try:
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine(c2, 5)
        assert e.value.code == fim.FIM_E_STATE
        bad = datagen.Csr(np.array([0, 2, 1], np.int64), np.array([0, 1], np.int32), 3)
        with pytest.raises(fim.FimError) as e:
            fim.fim_build_bitmaps(c2, bad.indptr, bad.indices, bad.m)
        assert e.value.code == fim.FIM_E_INVAL
        bad = datagen.Csr(np.array([0, 2], np.int64), np.array([0, 7], np.int32), 3)
        with pytest.raises(fim.FimError) as e:
            fim.fim_build_bitmaps(c2, bad.indptr, bad.indices, bad.m)
        assert e.value.code == fim.FIM_E_INVAL
        good = datagen.zipf_baskets(100, 10, 1.0, 3.0, 1)
        fim.fim_build_bitmaps(c2, good.indptr, good.indices, good.m)
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine(c2, 0)
        assert e.value.code == fim.FIM_E_INVAL
        fim.fim_mine(c2, 3)  # the ctx stays usable after errors
    finally:
        fim.fim_destroy(c2)


def test_empty_and_degenerate(ctx):
    for rows, m in [([], 5), ([[], [], []], 4), ([[0]], 1), ([[3]] * 10, 4)]:
        c = datagen.from_lists(rows, m)
        _same(ctx, c, 1)


@pytest.mark.slow
def test_quest_1M_full(ctx):
    c = datagen.quest_large()
    got = _same(ctx, c, 1000)
    assert len(got) == 34293


def test_planted_reduced_full(ctx):
    c = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    _same(ctx, c, 100)
