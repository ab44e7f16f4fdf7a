"""Compact CSR input (FIM_CSR_COMPACT: uint32 row offsets, uint16 item ids):
the same matrix as the wide CSR (int64 offsets, int32 ids), so every result
must equal the oracle's, bit for bit, on every input path -- single database
and batch; host pageable, page-locked (streamed or read in place) and device
arrays -- and a malformed compact CSR must be rejected like a wide one."""
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


def _compact(c):
    return datagen.Csr(indptr=c.indptr.astype(np.uint32), indices=c.indices.astype(np.uint16), m=c.m)


def _batch(seed, count):
    rng = np.random.default_rng(seed)
    dbs, ms = [], []
    for d in range(count):
        kind = d % 4
        if kind == 0:
            c = datagen.zipf_baskets(int(rng.integers(100, 5000)), int(rng.integers(5, 300)), 0.8, 6.0, [seed, d])
        elif kind == 1:
            c = datagen.random_dense(int(rng.integers(1, 400)), int(rng.integers(1, 12)), 0.5, [seed, d])
        elif kind == 2:
            c = datagen.from_lists([], int(rng.integers(1, 10)))          # no transactions
        else:
            c = datagen.planted(n=int(rng.integers(500, 3000)), m=int(rng.integers(20, 200)), n_patterns=5,
                                pat_len=(4, 7), frac=(0.02, 0.05), seed=[seed, d])
        dbs.append(c)
        ms.append(max(1, int(rng.integers(1, max(2, c.n // 20 + 2)))))
    return dbs, ms


def _check_batch(ctx, dbs, ms):
    for d, (c, m) in enumerate(zip(dbs, ms)):
        got = fim.fim_fetch_batched(ctx, d)
        assert got.sha256() == oracle.apriori(c.indptr, c.indices, c.m, m).sha256(), d


def _pinned_packed(dbs):
    """The compact CSRs packed back to back in page-locked host memory."""
    import torch
    ptr = torch.empty(sum(c.n + 1 for c in dbs), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    idx = torch.empty(max(1, sum(c.nnz for c in dbs)), dtype=torch.int16).pin_memory().numpy().view(np.uint16)
    out, po, io = [], 0, 0
    for c in dbs:
        ptr[po:po + c.n + 1] = c.indptr
        idx[io:io + c.nnz] = c.indices
        out.append(datagen.Csr(indptr=ptr[po:po + c.n + 1], indices=idx[io:io + c.nnz], m=c.m))
        po += c.n + 1
        io += c.nnz
    return out


@pytest.mark.parametrize("where", ["host", "pinned", "device"])
def test_single_database(ctx, where):
    import torch
    c = datagen.zipf_baskets(40_000, 700, 0.9, 7.0, [11])  # several build blocks, a ragged tail
    k = _compact(c)
    ip, ix = k.indptr, k.indices
    if where == "pinned":
        (kp,) = _pinned_packed([k])
        ip, ix = kp.indptr, kp.indices
    elif where == "device":
        ip = torch.from_numpy(ip.view(np.int32)).cuda()
        ix = torch.from_numpy(ix.view(np.int16)).cuda()
    fim.fim_build_bitmaps(ctx, ip, ix, c.m)
    for minsup in (60, 400):
        fim.fim_mine(ctx, minsup)
        assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(c.indptr, c.indices, c.m, minsup).sha256()


def test_single_database_largest_item_id(ctx):
    # ids up to 65,534 (n_items 65,535, the limit): the uint16 ids above
    # 32,767 must not be read as negative
    m = 65535
    rows = [[0, 40000, 65534], [40000, 65534], [65534], [0, 65534], []]
    c = datagen.from_lists(rows, m)
    k = _compact(c)
    fim.fim_build_bitmaps(ctx, k.indptr, k.indices, m)
    fim.fim_mine(ctx, 2)
    assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(c.indptr, c.indices, m, 2).sha256()


@pytest.mark.parametrize("streamed", [1, 0])
def test_batch_host_paths(ctx, streamed):
    dbs, ms = _batch(21, 28)
    kd = [_compact(c) for c in dbs]
    fim.fim_mine_batched(ctx, kd, ms)                  # pageable: staging copies
    _check_batch(ctx, dbs, ms)
    fim.fim_set_tuning(ctx, "batch_stream_copies", streamed)
    try:
        packed = _pinned_packed(kd)
        for seg in (0, 3):                             # automatic (eight) and three groups
            fim.fim_set_tuning(ctx, "batch_segments", seg)
            fim.fim_mine_batched(ctx, packed, ms)
            _check_batch(ctx, dbs, ms)
    finally:
        fim.fim_set_tuning(ctx, "batch_segments", 0)
        fim.fim_set_tuning(ctx, "batch_stream_copies", 1)


def test_batch_device_input_and_workload_sample(ctx):
    import torch

    class Dev:
        def __init__(self, c):
            k = _compact(c)
            ix = k.indices if c.nnz else np.zeros(1, np.uint16)
            self.indptr = torch.from_numpy(k.indptr.view(np.int32)).cuda()
            self.indices = torch.from_numpy(ix.view(np.int16)).cuda()
            self.m = c.m

    dbs, ms = _batch(22, 20)
    fim.fim_mine_batched(ctx, [Dev(c) for c in dbs], ms)
    _check_batch(ctx, dbs, ms)
    # the 4,096-database workload's size distribution, first 128 databases,
    # every one checked; then the same batch wide, which must agree
    specs = datagen.batched_specs(128)
    wl = [datagen.batched_db(s) for s in specs]
    wms = [datagen.minsup_from_ppm(c.n, 20_000) for c in wl]
    fim.fim_mine_batched(ctx, [Dev(c) for c in wl], wms)
    got = [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(wl))]
    for d, (c, m) in enumerate(zip(wl, wms)):
        assert got[d] == oracle.apriori(c.indptr, c.indices, c.m, m).sha256(), d
    fim.fim_mine_batched(ctx, wl, wms)
    assert [fim.fim_fetch_batched(ctx, d).sha256() for d in range(len(wl))] == got


def test_malformed_compact_rejected(ctx):
    good = datagen.zipf_baskets(3000, 50, 0.8, 5.0, [23])
    bad_id = datagen.Csr(np.array([0, 2, 3], np.uint32), np.array([1, 60, 2], np.uint16), 50)  # id 60 >= m
    bad_ptr = datagen.Csr(np.array([0, 3, 2], np.uint32), np.array([1, 2, 3], np.uint16), 50)  # decreasing
    for bad in (bad_id, bad_ptr):
        with pytest.raises(fim.FimError) as e:
            fim.fim_build_bitmaps(ctx, bad.indptr, bad.indices, bad.m)
        assert e.value.code == fim.FIM_E_INVAL
        with pytest.raises(fim.FimError) as e:
            fim.fim_mine_batched(ctx, [_compact(good), bad], [30, 1])
        assert e.value.code == fim.FIM_E_INVAL
    # the ctx still mines a valid compact input exactly afterwards
    k = _compact(good)
    fim.fim_build_bitmaps(ctx, k.indptr, k.indices, good.m)
    fim.fim_mine(ctx, 30)
    assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(good.indptr, good.indices, good.m, 30).sha256()
    fim.fim_mine_batched(ctx, [k, _compact(good)], [30, 45])
    _check_batch(ctx, [good, good], [30, 45])


@pytest.mark.parametrize("block", [16, 32, 64])
@pytest.mark.parametrize("coal", [1, 0])
def test_batch_build_shapes(ctx, block, coal):
    # every build block and both id-read orders on compact CSRs, with rows
    # long and short, empty rows and databases whose arrays start at odd
    # 16-bit offsets inside one buffer (the two-ids-per-load read meets
    # both alignments)
    rng = np.random.default_rng(block * 2 + coal)
    dbs, ms = [], []
    for d in range(14):
        rows = []
        for t in range(int(rng.integers(1, 2500))):
            k = int(rng.choice([0, 1, 2, 3, 5, 9, 40]))
            rows.append(sorted(rng.choice(120, size=min(k, 120), replace=False).tolist()))
        dbs.append(datagen.from_lists(rows, 120))
        ms.append(max(1, len(rows) // 15))
    packed = _pinned_packed([_compact(c) for c in dbs])
    fim.fim_set_tuning(ctx, "batch_build_block", block)
    fim.fim_set_tuning(ctx, "batch_build_coal", coal)
    try:
        for inp in (packed, [_compact(c) for c in dbs]):
            fim.fim_mine_batched(ctx, inp, ms, fim.FIM_MAXLEN(3))
            for d, (c, m) in enumerate(zip(dbs, ms)):
                got = fim.fim_fetch_batched(ctx, d)
                assert got.sha256() == oracle.apriori(c.indptr, c.indices, c.m, m, max_len=3).sha256(), d
    finally:
        fim.fim_set_tuning(ctx, "batch_build_block", 32)
        fim.fim_set_tuning(ctx, "batch_build_coal", 1)
