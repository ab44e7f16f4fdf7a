"""The Table 1 / Table 2 analogue columns of a mine (report.table_columns):
the average support of the frequent itemsets against the oracle's itemsets,
and the device memory the ctx reports holding against what the device
itself says was taken from it."""
import numpy as np
import pytest

import oracle
from paper_2412_19420_gb300 import datagen, report

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["grocery_like_10k_169", "quest_1M_1000"])
def test_average_support_matches_the_oracle_itemsets(name):
    gen, minsup = datagen.WORKLOADS[name]
    c = gen()
    ctx = fim.fim_create(0)
    try:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, minsup)
        got = fim.fim_fetch_results(ctx)
        cols = report.table_columns(got.supports, c.n, fim.fim_get_stats(ctx))
    finally:
        fim.fim_destroy(ctx)
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup)
    # Table 2: mean of S(X)/n over the frequent itemsets, in percent
    assert cols["frequent_itemsets"] == len(want)
    avg = 100.0 * float(np.mean(want.supports.astype(np.float64))) / c.n
    assert abs(cols["avg_support_pct"] - avg) <= 1e-12 * avg
    assert cols["avg_support_pct"] >= 100.0 * minsup / c.n


def test_peak_device_bytes_is_the_memory_the_ctx_holds():
    c = datagen.quest_large()
    # load every kernel module (and the library's static arrays) first, with
    # a ctx of its own, so that the measured ctx's drop is its own buffers
    warm = fim.fim_create(0)
    fim.fim_build_bitmaps(warm, c.indptr[:1001], c.indices[: int(c.indptr[1000])], c.m)
    fim.fim_mine(warm, 5)
    fim.fim_rules(warm, 500_000)
    fim.fim_destroy(warm)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx = fim.fim_create(0)
    try:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, 1000)
        st = fim.fim_get_stats(ctx)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        fim.fim_destroy(ctx)
    peak = st["peak_device_bytes"]
    # the bit columns alone: m columns of ceil(n/32) words
    assert peak >= 4 * c.m * ((c.n + 31) // 32)
    drop = free0 - free1
    # every byte the ctx counts was taken from the device (up to small
    # buffers the driver places in pages it already holds); what the device
    # lost beyond that is page rounding of the buffers, the ctx's streams,
    # events and captured graphs
    assert drop >= peak - (16 << 20), (drop, peak)
    assert drop <= peak + (256 << 20), (drop, peak)
