"""The batched pair pass on the tensor cores (the default) against the oracle
and against the CUDA-core tiles (FIM_PAIRS_POPC): databases whose frequent
items fill one 128 x 128 tile partly, exactly, or spill into several tiles
(off-diagonal ones included), ragged transaction counts, and launch shapes
that force many accumulator drains per tile and one CTA for every tile.
Also the batched build's blocks, with coalesced and lane-per-row id reads,
on ragged, long-row, packed and malformed CSRs."""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")


@pytest.fixture()
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _dense(n, m, p, seed):
    """n transactions over m items, each item present with probability p: with
    minsup 1 every item and pair is frequent, so m' = m."""
    rng = np.random.default_rng(seed)
    A = rng.random((n, m)) < p
    rows = [np.nonzero(r)[0].tolist() for r in A]
    return datagen.from_lists(rows, m)


def _pair_batch():
    # (n, m) pairs chosen so that m' = m crosses the tile edges 128 and 256
    shapes = [(1, 2), (37, 3), (129, 64), (1000, 127), (777, 128), (300, 129), (2049, 200),
              (513, 256), (260, 257), (131, 300), (4096, 130), (5, 400)]
    dbs = [_dense(n, m, 0.3, [7, i]) for i, (n, m) in enumerate(shapes)]
    return dbs, [1] * len(dbs)


def _check(ctx, dbs, ms, max_len):
    for d, (c, m) in enumerate(zip(dbs, ms)):
        got = fim.fim_fetch_batched(ctx, d)
        want = oracle.apriori(c.indptr, c.indices, c.m, m, max_len=max_len)
        assert got.sha256() == want.sha256(), (d, c.n, c.m, len(got), len(want))


@pytest.mark.parametrize("tuning", [{}, {"pairs_kdrain": 1}, {"pairs_kdrain": 3}, {"pairs_split": 1},
                                    {"pairs_split": 5, "pairs_kdrain": 2}])
def test_pairs_of_every_tile_shape(ctx, tuning):
    for k, v in tuning.items():
        fim.fim_set_tuning(ctx, k, v)
    dbs, ms = _pair_batch()
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_MAXLEN(2))
    assert fim.fim_get_stats(ctx)["pair_path"] == 1
    _check(ctx, dbs, ms, 2)


def test_tensor_and_cuda_core_pair_paths_agree(ctx):
    dbs, ms = _pair_batch()
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_MAXLEN(2))
    tc = [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(dbs))]
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_MAXLEN(2) | fim.FIM_PAIRS_POPC)
    assert fim.fim_get_stats(ctx)["pair_path"] == 0
    assert [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(dbs))] == tc


def test_full_mines_with_thresholds(ctx):
    # whole mines (pairs feed the prefix extension) on Zipf baskets whose
    # frequent items span one to three tiles
    dbs, ms = [], []
    for i, (n, m, ppm) in enumerate([(3000, 150, 20_000), (20_000, 400, 5_000), (700, 90, 50_000),
                                     (9000, 300, 4_000)]):
        c = datagen.zipf_baskets(n, m, 0.6, 9.0, [11, i])
        dbs.append(c)
        ms.append(datagen.minsup_from_ppm(c.n, ppm))
    fim.fim_set_tuning(ctx, "pairs_kdrain", 2)
    fim.fim_mine_batched(ctx, dbs, ms)
    _check(ctx, dbs, ms, 0)


@pytest.mark.parametrize("shape", range(7))
def test_every_pair_pass_shape_is_exact(ctx, shape):
    fim.fim_set_tuning(ctx, "batch_pairs_shape", shape)
    dbs, ms = _pair_batch()
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_MAXLEN(2))
    _check(ctx, dbs, ms, 2)


@pytest.mark.parametrize("block,coal", [(16, 1), (32, 1), (64, 1), (32, 0), (16, 0)])
def test_build_blocks_are_exact(ctx, block, coal):
    # ragged transaction counts around the 512 / 1,024 / 2,048-row blocks and
    # the 4,096-row column padding; duplicates and empty rows; rows long
    # enough that a warp reads its 32 rows' ids in several rounds of 256;
    # databases packed back to back, so that their item ids start at every
    # alignment
    fim.fim_set_tuning(ctx, "batch_build_block", block)
    fim.fim_set_tuning(ctx, "batch_build_coal", coal)
    rng = np.random.default_rng(block)
    dbs, ms = [], []
    for i, n in enumerate([1, 31, 511, 513, 1023, 1024, 1025, 2047, 2049, 4095, 4097, 9000]):
        m = int(rng.integers(3, 400))
        rows = [list(rng.integers(0, m, int(rng.integers(0, 9)))) for _ in range(n)]
        c = datagen.from_lists(rows, m)
        dbs.append(c)
        ms.append(max(1, n // 40))
    fim.fim_mine_batched(ctx, dbs, ms)
    _check(ctx, dbs, ms, 0)
    # long rows (pairs only: their supports depend on every bit's position)
    rng = np.random.default_rng(7)
    for i, (n, L, m) in enumerate([(700, 40, 450), (1500, 25, 300), (300, 90, 500), (2100, 12, 100)]):
        rows = [list(rng.integers(0, m, int(rng.integers(L // 2, 2 * L)))) for _ in range(n)]
        dbs.append(datagen.from_lists(rows, m))
        p = 1.25 * L / m
        ms.append(max(2, int(n * p * p / 2)))
    ptr = np.concatenate([c.indptr for c in dbs])
    idx = np.concatenate([c.indices for c in dbs])
    packed, po, io = [], 0, 0
    for c in dbs:
        packed.append(datagen.Csr(indptr=ptr[po:po + c.n + 1], indices=idx[io:io + c.nnz], m=c.m))
        po += c.n + 1
        io += c.nnz
    for batch in (dbs, packed):
        fim.fim_mine_batched(ctx, batch, ms, fim.FIM_MAXLEN(2))
        _check(ctx, dbs, ms, 2)


@pytest.mark.parametrize("block,coal", [(16, 1), (32, 1), (32, 0)])
def test_build_flags_malformed_rows(ctx, block, coal):
    # a row that ends before it starts, a row offset past the last id and an
    # item id out of range are each reported, whatever the block and build
    fim.fim_set_tuning(ctx, "batch_build_block", block)
    fim.fim_set_tuning(ctx, "batch_build_coal", coal)
    good = [datagen.zipf_baskets(3000, 100, 0.8, 6.0, [3, i]) for i in range(3)]
    bad = [datagen.Csr(np.array([0, 3, 1, 4], np.int64), np.array([0, 1, 2, 3], np.int32), 5),
           datagen.Csr(np.array([0, 9, 4], np.int64), np.array([0, 1, 2, 3], np.int32), 5),
           datagen.Csr(np.array([0, 2, 4], np.int64), np.array([0, 1, 7, 3], np.int32), 5)]
    for b in bad:
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine_batched(ctx, good[:1] + [b] + good[1:], [30, 1, 30, 30])
        assert e.value.code == fim.FIM_E_INVAL
    ms = [30] * len(good)
    fim.fim_mine_batched(ctx, good, ms)
    _check(ctx, good, ms, 0)


def test_autotuned_batch_shape_is_exact(ctx):
    from paper_2412_19420_gb300 import autotune
    dbs = [datagen.batched_db(s) for s in datagen.batched_specs(64)]
    ms = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    cfg, best_ms, table = autotune.tune_batched(ctx, dbs, ms, repeats=1)
    assert set(autotune.BATCH_SPACE) <= set(cfg) and best_ms > 0 and len(table) >= 2
    fim.fim_mine_batched(ctx, dbs, ms)
    _check(ctx, dbs, ms, 0)


@pytest.mark.parametrize("segments,group_dfs", [(1, 1), (2, 1), (3, 1), (8, 1), (8, 0)])
def test_pipelined_groups_are_exact(ctx, segments, group_dfs):
    # the batch graph pipelines groups of databases (build and rank of one
    # group beside the pair pass, root plan and prefix extension of the one
    # before, or the prefix extension once after all groups); any grouping
    # is exact, and so is a graph re-captured for another grouping
    fim.fim_set_tuning(ctx, "batch_segments", segments)
    fim.fim_set_tuning(ctx, "batch_group_dfs", group_dfs)
    dbs = [datagen.batched_db(s) for s in datagen.batched_specs(40, seed=5)]
    dbs[7] = datagen.from_lists([], 9)  # an empty database inside a group
    ms = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    for flags, ml in ((0, 0), (0, 0), (fim.FIM_STRICT, 0), (fim.FIM_MAXLEN(3), 3)):
        fim.fim_mine_batched(ctx, dbs, ms, flags)
        for d, (c, m) in enumerate(zip(dbs, ms)):
            want = oracle.apriori(c.indptr, c.indices, c.m, m, strict=bool(flags & fim.FIM_STRICT), max_len=ml)
            assert fim.fim_fetch_batched(ctx, d).sha256() == want.sha256(), (d, flags)


@pytest.mark.parametrize("pack", [1, 0])
def test_small_databases_packed_two_to_a_tile(ctx, pack):
    # databases with at most 64 frequent items share a tile pairwise (planned
    # on the device once m' is known): partners of unequal length, an odd one
    # out, databases without pairs in between, and larger ones mixed in
    fim.fim_set_tuning(ctx, "batch_pairs_pack", pack)
    rng = np.random.default_rng(21)
    dbs, ms = [], []
    for i in range(37):
        n = int(rng.integers(1, 6000))
        m = int(rng.choice([1, 2, 5, 33, 63, 64, 65, 90, 140]))
        dbs.append(_dense(n, m, float(rng.uniform(0.05, 0.3)), [31, i]))
        ms.append(max(1, n // int(rng.choice([4, 10, 50]))))
    for flags, ml in ((fim.FIM_MAXLEN(2), 2), (fim.FIM_MAXLEN(3), 3)):
        fim.fim_mine_batched(ctx, dbs, ms, flags)
        _check(ctx, dbs, ms, ml)
