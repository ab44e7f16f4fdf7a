"""Batched mining: many independent databases in one pass (one launch per
stage, build -> DFS replayed from a CUDA graph).  Every database's result
must equal the oracle's for that database alone, bit for bit."""
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


def _mixed_batch(seed, count):
    rng = np.random.default_rng(seed)
    dbs, ms = [], []
    for d in range(count):
        kind = d % 5
        if kind == 0:
            c = datagen.zipf_baskets(int(rng.integers(100, 5000)), int(rng.integers(5, 300)), 0.8, 6.0, [seed, d])
        elif kind == 1:
            c = datagen.random_dense(int(rng.integers(1, 400)), int(rng.integers(1, 12)), 0.5, [seed, d])
        elif kind == 2:
            c = datagen.from_lists([], int(rng.integers(1, 10)))          # no transactions
        elif kind == 3:
            c = datagen.planted(n=int(rng.integers(500, 3000)), m=int(rng.integers(20, 200)), n_patterns=5,
                                pat_len=(4, 7), frac=(0.02, 0.05), seed=[seed, d])
        else:
            c = datagen.from_lists([[0, 1, 2]] * int(rng.integers(1, 50)), 3)
        dbs.append(c)
        ms.append(max(1, int(rng.integers(1, max(2, c.n // 20 + 2)))))
    return dbs, ms


def _check_all(ctx, dbs, ms, strict=False, max_len=0):
    for d, (c, m) in enumerate(zip(dbs, ms)):
        got = fim.fim_fetch_batched(ctx, d)
        want = oracle.apriori(c.indptr, c.indices, c.m, m, strict=strict, max_len=max_len)
        assert got.sha256() == want.sha256(), (d, len(got), len(want))


def test_mixed_batch_matches_oracle(ctx):
    dbs, ms = _mixed_batch(1, 60)
    fim.fim_mine_batched(ctx, dbs, ms)
    _check_all(ctx, dbs, ms)


def test_graph_replay_and_new_shape(ctx):
    dbs, ms = _mixed_batch(2, 40)
    fim.fim_mine_batched(ctx, dbs, ms)
    first = [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(dbs))]
    fim.fim_mine_batched(ctx, dbs, ms)             # same shape: graph replay
    assert [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(dbs))] == first
    dbs2, ms2 = _mixed_batch(3, 25)                # new shape: new capture
    fim.fim_mine_batched(ctx, dbs2, ms2)
    _check_all(ctx, dbs2, ms2)


def test_descriptor_reuse_and_packed_host_input(ctx):
    # one descriptor table marshalled once and mined twice; the databases'
    # host arrays packed back to back (the library uploads them in one copy
    # per array)
    dbs, ms = _mixed_batch(4, 30)
    ptr = np.concatenate([c.indptr for c in dbs])
    idx = np.concatenate([c.indices for c in dbs])
    packed, po, io = [], 0, 0
    for c in dbs:
        packed.append(datagen.Csr(indptr=ptr[po:po + c.n + 1], indices=idx[io:io + c.nnz], m=c.m))
        po += c.n + 1
        io += c.nnz
    desc = fim.BatchDescriptor(packed, ms)
    for _ in range(2):
        fim.fim_mine_batched(ctx, desc)
        _check_all(ctx, dbs, ms)


def test_batch_flags(ctx):
    dbs, ms = _mixed_batch(4, 20)
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_STRICT)
    _check_all(ctx, dbs, ms, strict=True)
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_MAXLEN(2))
    _check_all(ctx, dbs, ms, max_len=2)
    fim.fim_mine_batched(ctx, dbs, ms, fim.FIM_DIFFSET_RULE)
    _check_all(ctx, dbs, ms)


def test_device_input(ctx):
    import torch

    class Dev:
        def __init__(self, c):
            self.indptr = torch.from_numpy(c.indptr).cuda()
            self.indices = torch.from_numpy(c.indices).cuda() if c.nnz else torch.zeros(1, dtype=torch.int32,
                                                                                           device="cuda")
            self.m = c.m

    dbs, ms = _mixed_batch(5, 15)
    fim.fim_mine_batched(ctx, [Dev(c) for c in dbs], ms)
    _check_all(ctx, dbs, ms)


def test_malformed_database_rejected(ctx):
    dbs, ms = _mixed_batch(6, 5)
    dbs[2] = datagen.Csr(np.array([0, 2], np.int64), np.array([0, 9], np.int32), 4)
    with pytest.raises(fim.FimError) as e:
        fim.fim_mine_batched(ctx, dbs, ms)
    assert e.value.code == fim.FIM_E_INVAL


def test_batched_workload_sample(ctx):
    # the 4,096-database workload's size distribution, first 256 databases
    specs = datagen.batched_specs(256)
    dbs = [datagen.batched_db(s) for s in specs]
    ms = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    fim.fim_mine_batched(ctx, dbs, ms)
    rng = np.random.default_rng(0)
    for d in rng.choice(len(dbs), 24, replace=False):
        got = fim.fim_fetch_batched(ctx, int(d))
        want = oracle.apriori(dbs[d].indptr, dbs[d].indices, dbs[d].m, ms[d])
        assert got.sha256() == want.sha256()


@pytest.mark.parametrize("streamed", [1, 0])
def test_pinned_host_input_read_in_place(ctx, streamed):
    # page-locked host CSRs packed back to back: uploaded group by group
    # inside the batch graph beside the earlier groups' mining (streamed), or
    # read over the host link in place by the build; a batch with one
    # pageable database among them goes up by staging copies instead -- all
    # exact
    import torch
    fim.fim_set_tuning(ctx, "batch_stream_copies", streamed)
    dbs, ms = _mixed_batch(7, 24)
    ptr = torch.from_numpy(np.concatenate([c.indptr for c in dbs])).pin_memory()
    idx = torch.from_numpy(np.concatenate([c.indices for c in dbs] + [np.zeros(1, np.int32)])).pin_memory()
    pn, inn = ptr.numpy(), idx.numpy()
    packed, po, io = [], 0, 0
    for c in dbs:
        packed.append(datagen.Csr(indptr=pn[po:po + c.n + 1], indices=inn[io:io + c.nnz], m=c.m))
        po += c.n + 1
        io += c.nnz
    for _ in range(2):
        fim.fim_mine_batched(ctx, packed, ms)
        _check_all(ctx, dbs, ms)
    mixed = list(packed)
    mixed[5] = dbs[5]  # pageable
    fim.fim_mine_batched(ctx, mixed, ms)
    _check_all(ctx, dbs, ms)
    for seg in (1, 3):  # explicit group counts
        fim.fim_set_tuning(ctx, "batch_segments", seg)
        fim.fim_mine_batched(ctx, packed, ms)
        _check_all(ctx, dbs, ms)
    fim.fim_set_tuning(ctx, "batch_segments", 0)
    fim.fim_set_tuning(ctx, "upload_mapped", 0)
    try:
        fim.fim_mine_batched(ctx, packed, ms)
        _check_all(ctx, dbs, ms)
    finally:
        fim.fim_set_tuning(ctx, "upload_mapped", 1)
        fim.fim_set_tuning(ctx, "batch_stream_copies", 1)


@pytest.mark.parametrize("warp_workers,ctas", [(1, 2), (1, 3), (0, 2)])
def test_warp_and_cta_workers_agree(ctx, warp_workers, ctas):
    # batches of short columns run the prefix extension with one warp per
    # worker; dense random databases give deep subtrees (long itemsets)
    fim.fim_set_tuning(ctx, "dfs_warp", warp_workers)
    fim.fim_set_tuning(ctx, "dfs_warp_ctas", ctas)
    try:
        dbs, ms = _mixed_batch(8, 45)
        for flags in (0, fim.FIM_STRICT, fim.FIM_MAXLEN(3)):
            fim.fim_mine_batched(ctx, dbs, ms, flags)
            _check_all(ctx, dbs, ms, strict=bool(flags & fim.FIM_STRICT), max_len=3 if flags >> 24 else 0)
    finally:
        fim.fim_set_tuning(ctx, "dfs_warp", 1)
        fim.fim_set_tuning(ctx, "dfs_warp_ctas", 2)


def test_single_mines_between_batches(ctx):
    # the same batch mined again after single-database mines (which reuse the
    # ctx's descriptor buffer) and after a larger batch: exact every time
    dbs, ms = _mixed_batch(9, 30)
    desc = fim.BatchDescriptor(dbs, ms)
    fim.fim_mine_batched(ctx, desc)
    _check_all(ctx, dbs, ms)
    c = dbs[3]
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, ms[3])
    assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(c.indptr, c.indices, c.m, ms[3]).sha256()
    fim.fim_mine_batched(ctx, desc)
    _check_all(ctx, dbs, ms)
    big, bms = _mixed_batch(10, 90)
    fim.fim_mine_batched(ctx, big, bms)
    _check_all(ctx, big, bms)
    fim.fim_mine_batched(ctx, desc)
    _check_all(ctx, dbs, ms)
