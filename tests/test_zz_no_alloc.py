"""The allocation-free entry point fim_pair_supports_noalloc, called through
the C ABI.  Its counts are compared exactly (integers) with two things that
share nothing with its kernels: numpy's int64 A^T A of the dense 0/1
transaction matrix (the diagonal is the column sums, Eq. 2 for a = b), and
the singleton and pair supports that the existing entry point fim_mine
reports for the same database.

The entry point exists for callers that cannot allocate device memory while
they use the library: a process whose own pool owns every device byte, or a
path that must not block in cudaMalloc/cudaFree.  Its scratch is a static
device array shared by every call.  This file is collected last so that a
failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
torch = pytest.importorskip("torch")


def _dense_ata(c):
    """Upper triangle (diagonal included) of A^T A for the de-duplicated 0/1
    matrix A[i, j] = 1 iff item j is in transaction i."""
    A = np.zeros((c.n, c.m), np.int64)
    rows = np.repeat(np.arange(c.n), np.diff(c.indptr))
    A[rows, c.indices] = 1
    return np.triu(A.T @ A).astype(np.uint32)


def _from_fim_mine(c):
    """Every singleton and pair with support >= 1, from fim_mine (minsup 1,
    itemsets of length <= 2)."""
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


def _noalloc(indptr, indices, m):
    ip = torch.from_numpy(indptr).cuda()
    ix = torch.from_numpy(indices if len(indices) else np.zeros(1, np.int32)).cuda()
    out = torch.full((m, m), 7, dtype=torch.int32, device="cuda")  # must be overwritten
    fim.fim_pair_supports_noalloc(ip, ix, m, out, torch.cuda.current_stream())
    return out.cpu().numpy().view(np.uint32)


def test_noalloc_matches_numpy_and_fim_mine_on_two_calls_in_a_row():
    # the second database is smaller, so stale scratch from the first call
    # would show up in its counts if a call left anything uncleared
    first = datagen.zipf_baskets(40_000, 300, 0.9, 7.0, 31)
    second = datagen.zipf_baskets(9_000, 70, 0.8, 5.0, 32)
    for c in (first, second):
        got = _noalloc(c.indptr, c.indices, c.m)
        want = _dense_ata(c)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got, _from_fim_mine(c))


def test_noalloc_duplicates_ragged_tail_and_empty_rows():
    # duplicated items collapse, empty transactions count toward n, and
    # n = 1,000 + 7 leaves a partly filled last word and tile
    rng = np.random.default_rng(5)
    n, m = 1007, 45
    lens = rng.integers(0, 9, n)
    lens[::13] = 0
    idx = rng.integers(0, m, int(lens.sum())).astype(np.int32)
    ip = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=ip[1:])
    c = datagen.Csr(indptr=ip, indices=idx, m=m)
    np.testing.assert_array_equal(_noalloc(ip, idx, m), _dense_ata(c))


def test_noalloc_empty_database():
    got = _noalloc(np.zeros(1, np.int64), np.zeros(0, np.int32), 5)
    np.testing.assert_array_equal(got, np.zeros((5, 5), np.uint32))


def test_noalloc_malformed_csr_is_rejected_and_the_next_call_is_exact():
    c = datagen.zipf_baskets(3_000, 40, 0.9, 5.0, 33)
    # an item id outside [0, n_items): every element index stays inside the
    # indices array, so the kernels read only valid memory and flag it
    bad_items = c.indices.copy()
    bad_items[len(bad_items) // 2] = c.m + 3
    # indptr decreasing in the middle, first and last entries intact
    bad_ptr = c.indptr.copy()
    bad_ptr[c.n // 2] = bad_ptr[c.n // 2 + 1] + 1
    for ip, ix in ((c.indptr, bad_items), (bad_ptr, c.indices)):
        with pytest.raises(fim.FimError) as e:
            _noalloc(ip, ix, c.m)
        assert e.value.code == fim.FIM_E_INVAL
        np.testing.assert_array_equal(_noalloc(c.indptr, c.indices, c.m), _dense_ata(c))


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
