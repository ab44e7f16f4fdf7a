"""Seeded synthetic transaction databases in CSR form.

Every workload the miner is measured or tested on is drawn here, from numpy's
``default_rng``, so that the GPU path and the CPU oracle see identical input.
This module only draws baskets: it contains no support counting, pruning or
itemset arithmetic, and it imports neither the oracle nor the GPU binding.

A database is a ``Csr`` with
  indptr  int64[n+1]  transaction i holds indices[indptr[i]:indptr[i+1]]
  indices int32[nnz]  item ids in [0, m)
and ``m`` items.  The generators emit each transaction's items distinct and
ascending, but the miner accepts duplicates (set semantics, Eq. 1).

Workload shapes (all stand-ins; the paper's own Groceries data is absent):
  grocery_like   n=10,000 x m=169, Zipf(1.0) popularity, Poisson(4.4) lengths
  quest          Agrawal-Srikant style pattern generator (c2 and c5 shapes)
  batched        4,096 independent Zipf(0.8) databases of uneven size
  planted        Zipf(1.1) background with embedded long correlated patterns
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np


@dataclasses.dataclass
class Csr:
    indptr: np.ndarray  # int64[n+1]
    indices: np.ndarray  # int32[nnz]
    m: int

    @property
    def n(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.m).tobytes())
        h.update(np.ascontiguousarray(self.indptr, dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.indices, dtype=np.int32).tobytes())
        return h.hexdigest()

    def row(self, i: int) -> np.ndarray:
        return self.indices[self.indptr[i]:self.indptr[i + 1]]


def _pairs_to_csr(rows: np.ndarray, items: np.ndarray, n: int, m: int) -> Csr:
    """Deduplicate (row, item) pairs and lay them out as a row-sorted CSR."""
    key = np.sort(rows.astype(np.int64) * m + items.astype(np.int64))
    if key.size > 1:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    r = key // m
    it = (key - r * m).astype(np.int32)
    counts = np.bincount(r, minlength=n).astype(np.int64)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return Csr(indptr, it, m)


def _zipf_weights(m: int, s: float) -> np.ndarray:
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


def _alias_table(weights: np.ndarray):
    """Walker's alias table (Vose's construction): draw i = floor(u * m), keep i
    if frac(u * m) < prob[i], else take alias[i]; P(j) = weights[j]."""
    m = weights.shape[0]
    scaled = weights * m / weights.sum()
    prob = np.ones(m)
    alias = np.arange(m)
    small = [i for i in range(m) if scaled[i] < 1.0]
    large = [i for i in range(m) if scaled[i] >= 1.0]
    while small and large:
        s, l = small.pop(), large.pop()
        prob[s] = scaled[s]
        alias[s] = l
        scaled[l] -= 1.0 - scaled[s]
        (small if scaled[l] < 1.0 else large).append(l)
    return prob, alias


def _alias_draw(rng, prob, alias, shape):
    u = rng.random(shape) * prob.shape[0]
    i = u.astype(np.int64)
    np.minimum(i, prob.shape[0] - 1, out=i)
    return np.where(u - i < prob[i], i, alias[i])


def _weighted_distinct_rows(rng, lengths: np.ndarray, weights: np.ndarray,
                            max_rounds: int = 64):
    """For row i draw lengths[i] DISTINCT indices with probability ~ weights.

    Sequential weighted draws with repeats rejected (the usual sampling
    without replacement): each row draws 2 L + 8 indices with replacement in
    one vectorised batch and keeps its first L distinct ones in draw order;
    rows still short draw again (rows left short after ``max_rounds`` are
    completed from the unused indices in weight order).
    Returns (rows, idx) arrays of equal length.
    """
    n = lengths.shape[0]
    m = weights.shape[0]
    prob, alias = _alias_table(weights)
    lengths = lengths.astype(np.int64)
    lmax = int(lengths.max()) if n else 0
    out = np.zeros((n, max(lmax, 1)), dtype=np.int64)   # kept indices, draw order
    cnt = np.zeros(n, dtype=np.int64)
    seen = np.zeros((n, (m + 63) // 64), dtype=np.uint64)
    todo = np.nonzero(lengths > 0)[0]
    for _ in range(max_rounds):
        if todo.size == 0:
            break
        need = lengths[todo] - cnt[todo]
        # enough draws for a typical row; the few rows still short draw again
        K = int(min(2 * need.max() + 8, 1.5 * need.mean() + 6))
        draws = _alias_draw(rng, prob, alias, (todo.size, K))
        for p in range(K):   # column by column: a row keeps a draw it has not seen yet
            idx = draws[:, p]
            word, bit = idx >> 6, (idx & 63).astype(np.uint64)
            sw = seen[todo, word]
            new = (((sw >> bit) & np.uint64(1)) == 0) & (cnt[todo] < lengths[todo])
            rows = todo[new]
            seen[rows, word[new]] = sw[new] | (np.uint64(1) << bit[new])
            out[rows, cnt[rows]] = idx[new]
            cnt[rows] += 1
        todo = todo[cnt[todo] < lengths[todo]]
    if todo.size:  # pathological (row length close to m): fill by weight order
        wo = np.argsort(-weights, kind="stable")
        for i in todo:
            cur = set(out[i, :cnt[i]].tolist())
            for j in wo:
                if cnt[i] == lengths[i]:
                    break
                if int(j) not in cur:
                    out[i, cnt[i]] = j
                    cnt[i] += 1
    keep = np.arange(out.shape[1])[None, :] < lengths[:, None]
    return np.nonzero(keep)[0].astype(np.int64), out[keep]


def zipf_baskets(n: int, m: int, s: float, mean_len: float, seed,
                 min_len: int = 1) -> Csr:
    """Baskets of distinct items; popularity Zipf(s) over a random rank->id map.

    Length of transaction i is max(min_len, Poisson(mean_len)), capped at m.
    Items are drawn without replacement with weight rank^-s; rank r maps to
    item id perm[r] for a seeded permutation, so ids carry no popularity order.
    """
    rng = np.random.default_rng(seed)
    lengths = np.minimum(np.maximum(min_len, rng.poisson(mean_len, n)), m)
    perm = rng.permutation(m)
    rows, ranks = _weighted_distinct_rows(rng, lengths, _zipf_weights(m, s))
    return _pairs_to_csr(rows, perm[ranks], n, m)


def grocery_like(seed: int = 0) -> Csr:
    """10,000 x 169, Zipf(1.0), Poisson(4.4) min 1: a stand-in for the shape of
    the retail basket data of the paper's experiments (Section IV.A)."""
    return zipf_baskets(10_000, 169, 1.0, 4.4, seed)


def quest(n: int, m: int, avg_len: float, avg_pat_len: float, n_patterns: int,
          seed, correlation: float = 0.5, corruption: float = 0.5,
          chunk: int = 1 << 18) -> Csr:
    """Pattern-based baskets in the style of Agrawal & Srikant's generator.

    * n_patterns "potential large itemsets": length max(1, Poisson(avg_pat_len));
      the first has uniform random items, each later one takes a fraction
      ~Exp(mean=correlation) of its items from its predecessor and the rest
      uniformly at random; pattern weights ~Exp(1), normalised.
    * transaction i has target length T_i = max(1, Poisson(avg_len)) and is
      filled with whole pattern draws (chosen by weight) until the running item
      total reaches the running target (so lengths track T_i within one draw).
    * corruption: from each drawn pattern, items are dropped one at a time
      while a uniform draw is below ``corruption`` (number dropped is geometric).
    Duplicates inside a transaction collapse.  A transaction whose draws were
    all fully corrupted stays empty, which the miner allows.
    """
    rng = np.random.default_rng(seed)
    plen = np.minimum(np.maximum(1, rng.poisson(avg_pat_len, n_patterns)), m)
    lmax = int(plen.max())
    pats = np.zeros((n_patterns, lmax), dtype=np.int64)
    prev = None
    for p in range(n_patterns):
        L = int(plen[p])
        chosen: list[int] = []
        if prev is not None:
            k = min(int(round(min(1.0, rng.exponential(correlation)) * L)), len(prev))
            if k:
                chosen = list(rng.choice(prev, size=k, replace=False))
        cs = set(chosen)
        while len(chosen) < L:
            j = int(rng.integers(m))
            if j not in cs:
                cs.add(j)
                chosen.append(j)
        pats[p, :L] = chosen
        prev = np.asarray(chosen, dtype=np.int64)
    wcdf = np.cumsum(rng.exponential(1.0, n_patterns))
    wcdf /= wcdf[-1]
    targets = np.maximum(1, rng.poisson(avg_len, n))
    slot = np.arange(lmax)[None, :]
    # expected kept length of one draw, to size the draw batch
    w = np.diff(np.concatenate([[0.0], wcdf]))
    q = corruption
    exp_keep = float(np.sum(w * (plen - q * (1 - q ** plen) / (1 - q)))) if q < 1 else 1.0
    exp_keep = max(exp_keep, 0.25)

    all_rows, all_items = [], []
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        tc = targets[r0:r1]
        cum_t = np.cumsum(tc)
        keep_l, item_l = [], []
        total = 0
        while total < cum_t[-1]:
            d = int((cum_t[-1] - total) / exp_keep * 1.15) + 64
            pid = np.searchsorted(wcdf, rng.random(d), side="right")
            np.minimum(pid, n_patterns - 1, out=pid)
            L = plen[pid]
            dropped = rng.geometric(1.0 - q, d) - 1 if q > 0 else np.zeros(d, np.int64)
            keep = np.maximum(L - dropped, 0)
            keys = rng.random((d, lmax), dtype=np.float32)
            keys[slot >= L[:, None]] = 2.0
            order = np.argsort(keys, axis=1, kind="stable")
            chosen = np.take_along_axis(pats[pid], order, axis=1)
            item_l.append(chosen[slot < keep[:, None]])
            keep_l.append(keep)
            total += int(keep.sum())
        keep = np.concatenate(keep_l)
        items = np.concatenate(item_l)
        cum_k = np.cumsum(keep)
        # last draw belonging to transaction t: first draw whose running total
        # reaches the running target
        last = np.searchsorted(cum_k, cum_t, side="left")
        first = np.concatenate([[0], last[:-1] + 1])
        ndraw = np.maximum(last - first + 1, 0)
        start_item = np.concatenate([[0], cum_k])[first]
        end_item = np.concatenate([[0], cum_k])[np.minimum(last + 1, len(cum_k))]
        end_item = np.where(ndraw > 0, end_item, start_item)
        cnt = end_item - start_item
        rows = np.repeat(np.arange(r0, r1, dtype=np.int64), cnt)
        offs = np.arange(int(cnt.sum()), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        all_rows.append(rows)
        all_items.append(items[np.repeat(start_item, cnt) + offs])
    return _pairs_to_csr(np.concatenate(all_rows), np.concatenate(all_items), n, m)


def quest_large(seed: int = 0) -> Csr:
    """1,000,000 x 1,000; avg length 10, 2,000 patterns of avg length 4."""
    return quest(1_000_000, 1000, 10.0, 4.0, 2000, seed)


def quest_stress(seed: int = 0) -> Csr:
    """10,000,000 x 5,000; avg length 12, 5,000 patterns of avg length 5."""
    return quest(10_000_000, 5000, 12.0, 5.0, 5000, seed)


def planted(n: int = 100_000, m: int = 2000, n_patterns: int = 500,
            pat_len=(6, 12), frac=(0.005, 0.03), zipf_s: float = 1.1,
            mean_len: float = 8.0, seed=0) -> Csr:
    """Zipf(s) background baskets plus embedded correlated patterns.

    Each pattern has a uniform length in [pat_len] of distinct random items and
    is inserted into a uniform random fraction in [frac] of the transactions
    (a random subset of rows).  Background lengths are max(1, Poisson(mean_len)).
    """
    rng = np.random.default_rng(seed)
    lengths = np.minimum(np.maximum(1, rng.poisson(mean_len, n)), m)
    perm = rng.permutation(m)
    rows, ranks = _weighted_distinct_rows(rng, lengths, _zipf_weights(m, zipf_s))
    rows_l, items_l = [rows], [perm[ranks]]
    for _ in range(n_patterns):
        L = int(rng.integers(pat_len[0], pat_len[1] + 1))
        items = rng.choice(m, size=L, replace=False)
        cnt = int(round(rng.uniform(frac[0], frac[1]) * n))
        sel = rng.choice(n, size=cnt, replace=False)
        rows_l.append(np.repeat(sel.astype(np.int64), L))
        items_l.append(np.tile(items.astype(np.int64), cnt))
    return _pairs_to_csr(np.concatenate(rows_l), np.concatenate(items_l), n, m)


@dataclasses.dataclass
class BatchSpec:
    n: int
    m: int
    seed: tuple


def batched_specs(n_db: int = 4096, seed: int = 0, log_n=(3.0, 5.0),
                  m_range=(64, 512)) -> list[BatchSpec]:
    """Sizes of the independent databases: n = floor(10^U(log_n)), m ~ U{m_range}."""
    out = []
    for d in range(n_db):
        rng = np.random.default_rng([seed, d])
        n = int(math.floor(10 ** rng.uniform(*log_n)))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        out.append(BatchSpec(n, m, (seed, d, 1)))
    return out


def batched_db(spec: BatchSpec, zipf_s: float = 0.8, mean_len: float = 6.0) -> Csr:
    """One database of the batched workload: Zipf(0.8), Poisson(6) min 1."""
    return zipf_baskets(spec.n, spec.m, zipf_s, mean_len, list(spec.seed))


def batched_dbs(specs, processes: int | None = None) -> list:
    """batched_db for every spec, in a spawn-context process pool (each
    database has its own seed, so the result does not depend on the pool)."""
    import multiprocessing as mp
    import os
    procs = processes or min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4)
    if procs <= 1 or len(specs) < 64:
        return [batched_db(s) for s in specs]
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            job = pool.map_async(batched_db, specs, chunksize=max(1, len(specs) // (4 * procs)))
            return job.get(timeout=900)
    except Exception:  # a pool that cannot start (e.g. no importable __main__): serial
        return [batched_db(s) for s in specs]


def minsup_from_ppm(n: int, ppm: int) -> int:
    """ceil(n * ppm / 1e6) in integers, at least 1 (threshold as a count)."""
    return max(1, (n * ppm + 999_999) // 1_000_000)


def random_dense(n: int, m: int, density: float, seed) -> Csr:
    """Independent Bernoulli(density) cells: small edge-case databases."""
    rng = np.random.default_rng(seed)
    dense = rng.random((n, m)) < density
    r, c = np.nonzero(dense)
    return _pairs_to_csr(r, c, n, m)


def from_lists(rows: list, m: int) -> Csr:
    """CSR from explicit transactions, keeping order and duplicates as given."""
    indptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=indptr[1:])
    flat = [int(x) for r in rows for x in r]
    return Csr(indptr, np.asarray(flat, dtype=np.int32), m)


# Named workloads: (generator, minsup as an absolute count)
WORKLOADS = {
    "grocery_like_10k_169": (grocery_like, 100),
    "quest_1M_1000": (quest_large, 1000),
    "planted_100k_2000": (lambda seed=0: planted(seed=seed), 500),
    "quest_10M_5000": (quest_stress, 5000),
}


# ---- seeded starting weights for the 8-64-64-2 scheduling MLP ----------
MLP_SHAPES = [(64, 8), (64,), (64, 64), (64,), (2, 64), (2,)]


def mlp_init_weights(seed: int = 0) -> np.ndarray:
    """Flat float32 vector W1,b1,W2,b2,W3,b3: He-uniform weights, zero biases."""
    rng = np.random.default_rng([seed, 8064642])
    parts = []
    for s in MLP_SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, s).ravel())
        else:
            parts.append(np.zeros(s[0]))
    return np.concatenate(parts).astype(np.float32)
