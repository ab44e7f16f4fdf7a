"""Launch-shape knobs and the autotuner.

A knob changes how the work is laid out on the GPU (worker width, workers per
SM, how deep a worker may hand prefixes to the queue, the pair pass split), never
what is computed: every shape must give the oracle's itemsets bit for bit.
"""
import json

import pytest

import oracle
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu
fim = pytest.importorskip("paper_2412_19420_gb300.fim")
autotune = pytest.importorskip("paper_2412_19420_gb300.autotune")


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


@pytest.fixture(scope="module")
def case():
    c = datagen.planted(n=20_000, m=600, n_patterns=40, seed=9)
    minsup = 120
    return c, minsup, oracle.apriori(c.indptr, c.indices, c.m, minsup).sha256()


SHAPES = [(256, 1, 0, 0), (256, 4, 8, 0), (512, 1, 2, 0), (512, 2, 6, 1), (256, 2, 1, 1), (256, 4, 8, 1)]


@pytest.mark.parametrize("threads,per_sm,split,reverse", SHAPES)
def test_every_shape_is_exact(ctx, case, threads, per_sm, split, reverse):
    c, minsup, want = case
    autotune.apply(ctx, {"dfs_threads": threads, "dfs_ctas_per_sm": per_sm, "split_depth": split,
                         "root_reverse": reverse})
    try:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, minsup)
        assert fim.fim_fetch_results(ctx).sha256() == want
        st = fim.fim_get_stats(ctx)
        assert st["dfs_workers"] > 0 and st["dfs_workers"] % per_sm == 0
        assert 0 <= st["dfs_busy_ns"] <= st["dfs_span_ns"] * st["dfs_workers"]
    finally:
        autotune.apply(ctx, autotune.DEFAULT)


def test_invalid_shapes_rejected(ctx):
    autotune.apply(ctx, autotune.DEFAULT)
    for key, v in [("dfs_threads", 384), ("dfs_threads", 128), ("dfs_ctas_per_sm", 0),
                   ("dfs_ctas_per_sm", 5), ("split_depth", 9)]:
        with pytest.raises(fim.FimError):
            fim.fim_set_tuning(ctx, key, v)
    with pytest.raises(fim.FimError):  # 512 x 4 > 1024 worker threads per SM
        fim.fim_set_tuning(ctx, "dfs_threads", 512)
    fim.fim_set_tuning(ctx, "dfs_ctas_per_sm", 1)
    fim.fim_set_tuning(ctx, "dfs_threads", 512)
    with pytest.raises(fim.FimError):
        fim.fim_set_tuning(ctx, "dfs_ctas_per_sm", 4)
    autotune.apply(ctx, autotune.DEFAULT)
    with pytest.raises(ValueError):
        autotune.apply(ctx, {"dfs_threads": 512, "dfs_ctas_per_sm": 4})


def test_autotune_picks_a_valid_shape_and_caches_it(ctx, case, tmp_path):
    c, minsup, want = case
    cache = str(tmp_path / "tune.json")
    space = {"dfs_threads": [256, 512], "dfs_ctas_per_sm": [2, 4], "split_depth": [4, 8]}
    best = autotune.tune(ctx, c, minsup, space=space, repeats=1, cache_path=cache)
    assert autotune.valid(best)
    with open(cache) as f:
        stored = json.load(f)
    assert len(stored) == 1 and next(iter(stored.values()))["dfs_threads"] == best["dfs_threads"]
    # a cache hit applies the stored choice without timing anything
    again = autotune.tune(ctx, c, minsup, space=space, repeats=1, cache_path=cache)
    assert again == best
    fim.fim_mine(ctx, minsup)
    assert fim.fim_fetch_results(ctx).sha256() == want
    autotune.apply(ctx, autotune.DEFAULT)


SPARSE_CASES = [
    ("planted", lambda: datagen.planted(n=20_000, m=600, n_patterns=40, seed=9), 120),
    ("zipf_deep", lambda: datagen.zipf_baskets(3000, 50, 0.8, 6.0, 9), 2),
    ("quest", lambda: datagen.quest(100_000, 300, 10.0, 4.0, 400, 5), 100),
]


@pytest.mark.parametrize("div", [-1, 0, 1, 2, 4, 64])
@pytest.mark.parametrize("name,gen,minsup", SPARSE_CASES, ids=[c[0] for c in SPARSE_CASES])
def test_sparse_classes_are_exact(ctx, name, gen, minsup, div):
    # sparse_div decides which class bitmaps are kept as their non-zero words;
    # dense, sparse and mixed stacks, counted dense or through diffsets, must
    # all give the oracle's itemsets
    c = gen()
    want = oracle.apriori(c.indptr, c.indices, c.m, minsup).sha256()
    fim.fim_set_tuning(ctx, "sparse_div", div)
    try:
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        for flags in (0, fim.FIM_DIFFSET_RULE, fim.FIM_NO_SPLIT):
            fim.fim_mine(ctx, minsup, flags)
            assert fim.fim_fetch_results(ctx).sha256() == want, flags
    finally:
        fim.fim_set_tuning(ctx, "sparse_div", -1)


@pytest.mark.parametrize("chunks,streams", [(1, 1), (3, 2), (4, 1), (16, 2)])
def test_chunked_host_upload_is_exact(ctx, chunks, streams):
    # the host CSR goes up in chunks of 512-transaction row blocks, each built
    # as it lands; ragged sizes leave a partial last block and empty chunks
    fim.fim_set_tuning(ctx, "upload_chunks", chunks)
    fim.fim_set_tuning(ctx, "upload_streams", streams)
    try:
        for n, m, thr in [(70_001, 200, 250), (1_500, 40, 10), (513, 9, 3)]:
            c = datagen.zipf_baskets(n, m, 0.9, 6.0, n)
            fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
            fim.fim_mine(ctx, thr)
            assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(c.indptr, c.indices, c.m, thr).sha256()
        # a malformed host CSR is still rejected, and the ctx stays usable
        c = datagen.zipf_baskets(5_000, 30, 0.9, 6.0, 1)
        bad = c.indptr.copy()
        bad[2600], bad[2601] = bad[2601], bad[2600] - 1  # not monotone
        with pytest.raises(fim.FimError):
            fim.fim_build_bitmaps(ctx, bad, c.indices, c.m)
        fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
        fim.fim_mine(ctx, 20)
        assert fim.fim_fetch_results(ctx).sha256() == oracle.apriori(c.indptr, c.indices, c.m, 20).sha256()
    finally:
        fim.fim_set_tuning(ctx, "upload_chunks", 4)
        fim.fim_set_tuning(ctx, "upload_streams", 2)
    for key, v in (("upload_chunks", 0), ("upload_chunks", 17), ("upload_streams", 3)):
        with pytest.raises(fim.FimError):
            fim.fim_set_tuning(ctx, key, v)


def test_cluster_sort_equals_launch_sequence(ctx):
    # outputs from a handful of sets to tens of thousands, both compaction
    # paths, oracle-exact: 3,265 and 10,275 sets (one key word), 35,517 (one
    # word, 16 CTAs of ~2,220), 51,640 (three words, 16 x 3,228 of a 3,936
    # capacity), and 96,497 / 405,597 sets that exceed one cluster
    plant = datagen.planted(n=20_000, m=800, n_patterns=60, seed=4)
    cases = [(datagen.from_lists([[0, 1], [1, 2], [0, 1, 2]] * 3, 3), 2),
             (datagen.zipf_baskets(4_097, 130, 0.9, 6.0, 2), 12),
             (datagen.zipf_baskets(70_001, 200, 0.9, 6.0, 3), 60),
             (datagen.zipf_baskets(200_000, 300, 0.8, 8.0, 5), 100),
             (plant, 400), (plant, 300),
             (datagen.planted(n=20_000, m=600, n_patterns=40, seed=9), 120)]
    try:
        for c, thr in cases:
            want = oracle.apriori(c.indptr, c.indices, c.m, thr).sha256()
            fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
            for on in (1, 0, 1):
                fim.fim_set_tuning(ctx, "compact_cluster", on)
                fim.fim_mine(ctx, thr)
                assert fim.fim_fetch_results(ctx).sha256() == want, (c.n, thr, on)
    finally:
        fim.fim_set_tuning(ctx, "compact_cluster", 1)


def test_mapped_host_input_is_exact(ctx):
    # page-locked host CSR: read in place by the build kernel (upload_mapped 1)
    # or staged by copies (0); pageable numpy arrays always take the copies
    torch = pytest.importorskip("torch")
    try:
        for n, m, thr in [(70_001, 200, 250), (513, 9, 3)]:
            c = datagen.zipf_baskets(n, m, 0.9, 6.0, n + 1)
            want = oracle.apriori(c.indptr, c.indices, c.m, thr).sha256()
            ip = torch.from_numpy(c.indptr).pin_memory()
            ix = torch.from_numpy(c.indices).pin_memory()
            for mapped in (1, 0):
                fim.fim_set_tuning(ctx, "upload_mapped", mapped)
                for src in ((ip.numpy(), ix.numpy()), (c.indptr, c.indices)):
                    fim.fim_build_bitmaps(ctx, src[0], src[1], c.m)
                    fim.fim_mine(ctx, thr)
                    assert fim.fim_fetch_results(ctx).sha256() == want
        # a malformed pinned CSR is rejected in place too
        c = datagen.zipf_baskets(5_000, 30, 0.9, 6.0, 2)
        bad = torch.from_numpy(c.indptr.copy()).pin_memory()
        bad[3000], bad[3001] = int(bad[3001]), int(bad[3000]) - 1
        fim.fim_set_tuning(ctx, "upload_mapped", 1)
        with pytest.raises(fim.FimError):
            fim.fim_build_bitmaps(ctx, bad.numpy(), torch.from_numpy(c.indices).pin_memory().numpy(), c.m)
    finally:
        fim.fim_set_tuning(ctx, "upload_mapped", 1)


def test_probes_are_plausible(ctx):
    # measurement probes: the AND/popc word-pair rate and the L2 read
    # bandwidth of the GPU (GB300: 152 SMs near 2 GHz, L2 well above HBM),
    # and the tcgen05 f8f6f4 MMA rate (dense fp8 nominal 4.5 PFLOP/s)
    popc = fim.fim_probe(ctx, 0)
    l2 = fim.fim_probe(ctx, 1)
    assert 1e11 < popc < 1e14
    assert 1000 < l2 < 200_000
    mma = [fim.fim_probe(ctx, w) for w in (2, 3, 4, 5)]
    assert all(100 < t < 6000 for t in mma), mma
    # A from tensor memory is the fastest form, and N = 64 the slowest
    assert mma[0] >= mma[1] and mma[3] <= mma[2]
    with pytest.raises(fim.FimError):
        fim.fim_probe(ctx, 6)
