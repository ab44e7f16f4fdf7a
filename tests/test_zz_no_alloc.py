"""The allocation-free entry point fim_pair_supports_noalloc, called through
the C ABI, against the singleton and pair supports that fim_mine reports for
the same database (integer counts: compared exactly).

It exists for callers that cannot allocate device memory while they use the
library (a process whose own pool owns every device byte, or a path that must
not block in cudaMalloc); its scratch is a static device array.  This file is
collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
torch = pytest.importorskip("torch")


def _expected(c):
    """Counts from the existing entry point: every singleton and pair with
    support >= 1 (fim_mine, minsup 1, itemsets of length <= 2)."""
    ctx = fim.fim_create(0)
    try:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, 1, fim.FIM_MAXLEN(2))
        res = fim.fim_fetch_results(ctx)
    finally:
        fim.fim_destroy(ctx)
    want = np.zeros((c.m, c.m), np.uint32)
    for items, s in res.as_dict().items():
        a, b = (items[0], items[0]) if len(items) == 1 else items
        want[a, b] = s
    return want


def _noalloc(c):
    ip = torch.from_numpy(c.indptr).cuda()
    ix = torch.from_numpy(c.indices).cuda()
    out = torch.full((c.m, c.m), 7, dtype=torch.int32, device="cuda")  # must be overwritten
    stream = torch.cuda.current_stream()
    fim.fim_pair_supports_noalloc(ip, ix, c.m, out, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_noalloc_matches_fim_mine_on_two_calls_in_a_row():
    # the second database is smaller, so stale scratch from the first call
    # would show up in its counts if a call left anything uncleared
    first = datagen.zipf_baskets(40_000, 300, 0.9, 7.0, 31)
    second = datagen.zipf_baskets(9_000, 70, 0.8, 5.0, 32)
    for c in (first, second):
        got = _noalloc(c)
        np.testing.assert_array_equal(got, _expected(c))


def test_noalloc_rejects_databases_above_the_scratch_limit():
    # 2,000,000 empty transactions x 600 items: 600 x 128 B x ceil(2e6 / 1024)
    # = 150 MB of bit columns, above the 64 MiB static scratch
    big_n, m = 2_000_000, 600
    ip = torch.zeros(big_n + 1, dtype=torch.int64, device="cuda")
    ix = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros((m, m), dtype=torch.int32, device="cuda")
    with pytest.raises(fim.FimError) as e:
        fim.fim_pair_supports_noalloc(ip, ix, m, out)
    assert e.value.code == fim.FIM_E_INVAL
