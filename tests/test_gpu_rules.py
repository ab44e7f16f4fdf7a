"""GPU association rules vs the oracle: bit-exact rule lists.

The miner and fim_rules run on the GPU through the C ABI; the oracle mines the
same seeded database on the CPU and derives its rules from its own itemsets.
Set indices and antecedent masks must match exactly, and conf / lift bit for
bit (both sides divide the same integers once, correctly rounded).
"""
import numpy as np
import pytest

import oracle
from oracle import rules as orules
from paper_2412_19420_gb300 import datagen

pytestmark = pytest.mark.gpu

fim = pytest.importorskip("paper_2412_19420_gb300.fim")


@pytest.fixture(scope="module")
def ctx():
    c = fim.fim_create(0)
    yield c
    fim.fim_destroy(c)


def _gpu_rules(ctx, c, minsup, ppm, max_len=0, flags=0):
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, minsup, flags)
    n = fim.fim_rules(ctx, ppm, max_len)
    r = fim.fim_fetch_rules(ctx)
    assert len(r) == n
    return r


def _want(c, minsup, ppm, max_len=0, strict=False, set_max_len=0):
    its = oracle.apriori(c.indptr, c.indices, c.m, minsup, strict=strict, max_len=set_max_len)
    return orules.rules(its, len(c.indptr) - 1, ppm, max_len)


def _same(got, want):
    assert len(got) == len(want), f"{len(got)} vs {len(want)} rules"
    assert np.array_equal(got.set_index, want.set_index)
    assert np.array_equal(got.ante_mask, want.ante_mask)
    assert np.array_equal(got.conf.view(np.uint64), want.conf.view(np.uint64))
    assert np.array_equal(got.lift.view(np.uint64), want.lift.view(np.uint64))


@pytest.mark.parametrize("seed", range(4))
def test_random_small(ctx, seed):
    rng = np.random.default_rng(70 + seed)
    n, m = int(rng.integers(10, 400)), int(rng.integers(3, 12))
    c = datagen.random_dense(n, m, float(rng.uniform(0.2, 0.8)), [seed, 5])
    thr = int(rng.integers(1, max(2, n // 6)))
    for ppm in (0, 1, 333_333, 500_000, 1_000_000):
        _same(_gpu_rules(ctx, c, thr, ppm), _want(c, thr, ppm))


def test_max_len_and_mine_flags(ctx):
    c = datagen.random_dense(300, 10, 0.55, 17)
    for ml in (2, 3, 7, 20):
        _same(_gpu_rules(ctx, c, 20, 250_000, max_len=ml), _want(c, 20, 250_000, max_len=ml))
    # strict threshold and a bounded itemset length still give downward-closed sets
    _same(_gpu_rules(ctx, c, 20, 250_000, flags=fim.FIM_STRICT), _want(c, 20, 250_000, strict=True))
    _same(_gpu_rules(ctx, c, 20, 250_000, flags=fim.FIM_MAXLEN(3)), _want(c, 20, 250_000, set_max_len=3))


def test_long_sets_and_many_warps(ctx):
    # all-ones over 12 items: 4,095 sets (512 CTAs of 8 warps), sets up to
    # 12 items (4,094 antecedents each, 128 ballot rounds), 523,250 rules
    m, n = 12, 40
    c = datagen.from_lists([list(range(m))] * n, m)
    got = _gpu_rules(ctx, c, n, 1_000_000)
    assert len(got) == 3**m - 2 ** (m + 1) + 1
    _same(got, _want(c, n, 1_000_000))


def test_many_sets_few_candidates(ctx):
    # every subset of 14 items once: 16,383 frequent sets (two scan chunks of
    # set counts); max_len 2 leaves 182 candidate rules, all with conf 1/2
    m = 14
    c = datagen.from_lists([[j for j in range(m) if i >> j & 1] for i in range(1 << m)], m)
    got = _gpu_rules(ctx, c, 1, 0, max_len=2)
    assert fim.fim_rules_evaluated(ctx) == 2 * 91
    assert set(got.conf.tolist()) == {0.5} and set(got.lift.tolist()) == {1.0}
    _same(got, _want(c, 1, 0, max_len=2))


def test_evaluated_count(ctx):
    c = datagen.random_dense(250, 11, 0.5, 21)
    _gpu_rules(ctx, c, 15, 700_000)
    its = oracle.apriori(c.indptr, c.indices, c.m, 15)
    L = np.diff(its.offsets.astype(np.int64))
    assert fim.fim_rules_evaluated(ctx) == int(((np.int64(1) << L[L >= 2]) - 2).sum())


def test_zipf_tiles_and_ragged(ctx):
    for n, m, s in [(4097, 130, 2), (70_001, 200, 3)]:
        c = datagen.zipf_baskets(n, m, 0.9, 6.0, s)
        thr = max(2, n // 300)
        for ppm in (100_000, 600_000):
            _same(_gpu_rules(ctx, c, thr, ppm), _want(c, thr, ppm))


def test_device_output_and_states(ctx):
    torch = pytest.importorskip("torch")
    c = datagen.random_dense(200, 9, 0.5, 8)
    want = _want(c, 10, 400_000)
    fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
    fim.fim_mine(ctx, 10)
    with pytest.raises(fim.FimError):  # no rules built for this mine yet
        fim.fim_fetch_rules(ctx)
    n = fim.fim_rules(ctx, 400_000)
    d = torch.device("cuda", 0)
    out = (torch.empty(n, dtype=torch.int64, device=d), torch.empty(n, dtype=torch.int32, device=d),
           torch.empty(n, dtype=torch.float64, device=d), torch.empty(n, dtype=torch.float64, device=d))
    r = fim.fim_fetch_rules(ctx, out)
    host = fim.Rules(r.set_index.cpu().numpy().view(np.uint64), r.ante_mask.cpu().numpy().view(np.uint32),
                     r.conf.cpu().numpy(), r.lift.cpu().numpy())
    _same(host, want)
    small = tuple(np.empty(max(1, n - 1), dt) for dt in (np.uint64, np.uint32, np.float64, np.float64))
    with pytest.raises(fim.FimError) as e:
        fim.fim_fetch_rules(ctx, small)
    assert e.value.args[0].endswith(f"({fim.FIM_E_TOO_SMALL})")
    for bad in ((1_000_001, 0), (0, 1), (0, 21), (0, -1)):
        with pytest.raises(fim.FimError):
            fim.fim_rules(ctx, *bad)
    fim.fim_mine(ctx, 11)  # a new mine invalidates the rules
    with pytest.raises(fim.FimError):
        fim.fim_fetch_rules(ctx)


def test_empty_outputs(ctx):
    c = datagen.from_lists([[i] for i in range(6)], 6)
    assert len(_gpu_rules(ctx, c, 1, 0)) == 0
    c = datagen.from_lists([[0, 1]] * 3, 4)
    assert len(_gpu_rules(ctx, c, 4, 0)) == 0  # nothing frequent
    got = _gpu_rules(ctx, c, 3, 0)
    _same(got, _want(c, 3, 0))
    assert got.ante_mask.tolist() == [1, 2] and got.lift.tolist() == [1.0, 1.0]


@pytest.mark.slow
def test_quest_1M_rules(ctx):
    # the 10^6 x 1,000 Quest-style workload at minsup 1,000, 50% confidence
    c = datagen.quest_large()
    _same(_gpu_rules(ctx, c, 1000, 500_000), _want(c, 1000, 500_000))
