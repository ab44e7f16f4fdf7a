"""Split mines on one GPU: the shards of a database, mined one after another
through fim_mine_shard, are disjoint, and fim_merge_results of their parts
is bit-identical to the oracle's answer (and to fim_mine's).
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


def _parts(ctx, c, minsup, n_shards, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    parts = []
    for s in range(n_shards):
        fim.fim_mine_shard(ctx, minsup, flags, s, n_shards)
        parts.append(fim.fim_fetch_results(ctx))
    return parts


def _check_split(ctx, c, minsup, n_shards, flags=0, strict=False, max_len=0):
    parts = _parts(ctx, c, minsup, n_shards, flags)
    seen = {}
    for s, p in enumerate(parts):
        for x in p.as_dict():
            assert x not in seen, f"{x} in shards {seen[x]} and {s}"
            seen[x] = s
            assert s == 0 or len(x) > 2, "a shard > 0 reported a singleton or pair"
    fim.fim_merge_results(ctx, len(c.indptr) - 1, c.m, parts)
    got = fim.fim_fetch_results(ctx)
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup, strict=strict, max_len=max_len)
    assert got.sha256() == want.sha256()
    return parts


@pytest.mark.parametrize("n_shards", [1, 2, 3, 8])
def test_split_zipf_and_dense(ctx, n_shards):
    _check_split(ctx, datagen.zipf_baskets(20_000, 150, 0.9, 6.0, 5), 40, n_shards)
    _check_split(ctx, datagen.random_dense(300, 12, 0.55, 6), 20, n_shards)


def test_split_planted_and_flags(ctx):
    c = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    parts = _check_split(ctx, c, 100, 4)
    # dealing the root classes round-robin balances the work: no shard holds
    # far more than a quarter of the sets of size >= 3 (contiguous ranges of
    # equal estimated cost gave one shard 55% on this workload)
    deep = [sum(len(x) > 2 for x in p.as_dict()) for p in parts]
    assert max(deep) <= 0.35 * sum(deep), deep
    z = datagen.zipf_baskets(5000, 60, 0.8, 6.0, 3)
    _check_split(ctx, z, 10, 3, flags=fim.FIM_STRICT, strict=True)
    _check_split(ctx, z, 10, 3, flags=fim.FIM_MAXLEN(3), max_len=3)
    _check_split(ctx, z, 10, 5, flags=fim.FIM_PAIRS_POPC)
    _check_split(ctx, z, 10, 2, flags=fim.FIM_NO_SPLIT)


def test_more_shards_than_classes(ctx):
    c = datagen.from_lists([[0, 1, 2]] * 5 + [[3, 4]] * 5, 5)
    parts = _check_split(ctx, c, 5, 16)
    # {0,1,2} with its 6 nonempty proper subsets, {3,4} with its 2 items
    assert sum(len(p) for p in parts) == 10


def test_merge_device_parts_and_rules(ctx):
    torch = pytest.importorskip("torch")
    c = datagen.zipf_baskets(30_000, 120, 0.9, 6.0, 8)
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, 60)
    want = fim.fim_fetch_results(ctx)
    fim.fim_rules(ctx, 300_000)
    want_rules = fim.fim_fetch_rules(ctx)
    d = torch.device("cuda", 0)
    parts = []
    for s in range(3):
        fim.fim_mine_shard(ctx, 60, 0, s, 3)
        p = fim.fim_fetch_results(ctx)
        parts.append(tuple(torch.from_numpy(a.view({8: np.int64, 4: np.int32}[a.itemsize])).to(d)
                           for a in (p.offsets, p.items, p.supports)))
    fim.fim_merge_results(ctx, len(c.indptr) - 1, c.m, parts)
    assert fim.fim_fetch_results(ctx).sha256() == want.sha256()
    fim.fim_rules(ctx, 300_000)
    r = fim.fim_fetch_rules(ctx)
    assert np.array_equal(r.set_index, want_rules.set_index) and np.array_equal(r.ante_mask, want_rules.ante_mask)
    assert np.array_equal(r.conf.view(np.uint64), want_rules.conf.view(np.uint64))
    assert np.array_equal(r.lift.view(np.uint64), want_rules.lift.view(np.uint64))


def test_merge_rejects_malformed_parts(ctx):
    ok = (np.array([0, 1, 3], np.uint64), np.array([2, 0, 4], np.uint32), np.array([9, 5], np.uint32))
    fim.fim_merge_results(ctx, 10, 5, [ok])
    got = fim.fim_fetch_results(ctx)
    assert got.as_dict() == {(2,): 9, (0, 4): 5}
    bad_item = (ok[0], np.array([2, 0, 5], np.uint32), ok[2])
    bad_off = (np.array([0, 2, 1], np.uint64), ok[1], ok[2])
    bad_empty = (np.array([0, 1, 1], np.uint64), ok[1][:1], ok[2])  # a set with no item
    for parts in ([bad_item], [bad_off], [bad_empty], [ok, bad_item]):
        with pytest.raises(fim.FimError):
            fim.fim_merge_results(ctx, 10, 5, parts)
    for bad in ((-1, 5), (10, 70_000)):
        with pytest.raises(fim.FimError):
            fim.fim_merge_results(ctx, bad[0], bad[1], [ok])
    for s, n in ((2, 2), (-1, 2), (0, 0), (0, 2000)):
        with pytest.raises(fim.FimError):
            fim.fim_mine_shard(ctx, 1, 0, s, n)


def test_mine_sharded_one_rank_nccl(ctx):
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    from paper_2412_19420_gb300 import shard
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        c = datagen.zipf_baskets(20_000, 100, 0.9, 6.0, 12)
        ip = torch.from_numpy(c.indptr).cuda()
        ix = torch.from_numpy(c.indices).cuda()
        n = shard.mine_sharded(ctx, ip, ix, c.m, 40)
        got = fim.fim_fetch_results(ctx)
        want = oracle.apriori(c.indptr, c.indices, c.m, 40)
        assert n == len(want) and got.sha256() == want.sha256()
    finally:
        dist.destroy_process_group()
