"""Autotuner for the miner's launch shapes (fim_set_tuning knobs).

For one workload it times every candidate configuration with CUDA events on
the miner's stream (median of `repeats` mines after one warm-up) and keeps
the fastest.  Knobs only change scheduling and tile shapes, never results.
Choices are cached in a JSON file keyed by a workload signature.

    cfg = autotune.tune(ctx, csr, minsup)          # or tune_batched(ctx, dbs, minsups)
    autotune.apply(ctx, cfg)
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

from . import fim

SPACE = {
    "dfs_threads": [256, 512],
    "dfs_ctas_per_sm": [2, 4],
    "split_depth": [4, 8],
    "sparse_div": [-1, 0, 4],
}
DEFAULT = {"dfs_threads": 256, "dfs_ctas_per_sm": 4, "split_depth": 8, "sparse_div": -1,
           "root_reverse": 0, "pairs_kdrain": 0, "pairs_split": 0}
# a batch: the tensor-core pair pass's launch shape (ring stages, raw-bit
# staging depth, CTAs per SM), the build's words per column and CTA, and the
# DFS workers; searched one knob at a time from BATCH_DEFAULT
BATCH_SPACE = {
    "batch_pairs_shape": [0, 1, 2, 3, 4, 5, 6],
    "batch_build_block": [16, 32, 64],
    "dfs_ctas_per_sm": [2, 4],
    "split_depth": [4, 8],
    "dfs_warp_ctas": [2, 3],
}
BATCH_DEFAULT = dict(DEFAULT, batch_pairs_shape=0, batch_build_block=32, batch_segments=0, dfs_warp_ctas=2)


def valid(cfg: dict) -> bool:
    """A DFS worker is register-capped so that at most 1024 worker threads fit an SM."""
    return cfg.get("dfs_threads", 512) * cfg.get("dfs_ctas_per_sm", 1) <= 1024


def signature(kind: str, n: int, m: int, nnz: int, minsup, flags: int) -> str:
    """Bucketed workload signature: log2 sizes, so nearby workloads share a choice."""
    def lg(v):
        return int(v).bit_length()
    return f"{kind}:n{lg(n)}:m{lg(m)}:z{lg(nnz)}:s{lg(minsup)}:f{int(flags)}"


def apply(ctx, cfg: dict) -> None:
    if not valid(cfg):
        raise ValueError(f"invalid launch shape {cfg}")
    # one worker per SM first, so that no intermediate (threads, ctas) pair
    # exceeds an SM while the shape changes
    fim.fim_set_tuning(ctx, "dfs_ctas_per_sm", 1)
    for k in sorted(cfg, key=lambda k: k == "dfs_ctas_per_sm"):
        fim.fim_set_tuning(ctx, k, int(cfg[k]))


def _time_ms(run, repeats: int) -> float:
    import torch
    ts = []
    for i in range(repeats + 1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        if i:
            ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _search(ctx, run, space, repeats):
    keys = sorted(space)
    best, best_ms, table = None, float("inf"), []
    for vals in itertools.product(*(space[k] for k in keys)):
        cfg = dict(DEFAULT, **dict(zip(keys, vals)))
        if not valid(cfg):
            continue
        apply(ctx, cfg)
        ms = _time_ms(run, repeats)
        table.append((cfg, ms))
        if ms < best_ms:
            best, best_ms = cfg, ms
    apply(ctx, best)
    return best, best_ms, table


def _coordinate_search(ctx, run, space, start, repeats, sweeps=2):
    """One knob at a time: each value of each knob with the others held, a
    change kept when it is at least 1% faster; up to `sweeps` passes."""
    cur = dict(start)
    apply(ctx, cur)
    best_ms = _time_ms(run, repeats)
    table = [(dict(cur), best_ms)]
    for _ in range(sweeps):
        improved = False
        for k in sorted(space):
            for v in space[k]:
                if v == cur.get(k):
                    continue
                cfg = dict(cur, **{k: v})
                if not valid(cfg):
                    continue
                apply(ctx, cfg)
                ms = _time_ms(run, repeats)
                table.append((cfg, ms))
                if ms < 0.99 * best_ms:
                    cur, best_ms, improved = cfg, ms, True
        if not improved:
            break
    apply(ctx, cur)
    return cur, best_ms, table


def _cached(cache_path, sig):
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            return json.load(f).get(sig)
    return None


def _store(cache_path, sig, cfg, ms):
    if not cache_path:
        return
    data = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            data = json.load(f)
    data[sig] = dict(cfg, _ms=ms)
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)


def tune(ctx, csr, minsup: int, flags: int = 0, space=None, repeats: int = 3, cache_path: str | None = None):
    """Best knob setting for one database; the miner's stream is the default
    stream's peer (fim_create without a stream), timed with device events
    around whole mines."""
    sig = signature("single", csr.n, csr.m, csr.nnz, minsup, flags)
    hit = _cached(cache_path, sig)
    if hit:
        cfg = {k: v for k, v in hit.items() if not k.startswith("_")}
        apply(ctx, cfg)
        return cfg
    fim.fim_build_bitmaps(ctx, csr.indptr, csr.indices, csr.m)

    def run():
        fim.fim_mine(ctx, minsup, flags)

    best, ms, _ = _search(ctx, run, space or SPACE, repeats)
    _store(cache_path, sig, best, ms)
    return best


def tune_batched(ctx, dbs, minsups, flags: int = 0, space=None, repeats: int = 2,
                 cache_path: str | None = None, desc=None):
    """Best knob setting for a batch: the tensor-core pair pass's launch shape,
    the build's block, the DFS workers and split depth (BATCH_SPACE), by a
    coordinate search timed around whole batched mines.  dbs/minsups give the
    workload signature; `desc` (a fim.BatchDescriptor of the same batch, host
    or device arrays) is what is mined, else dbs/minsups themselves.
    Returns (config, ms of the best config, table of (config, ms))."""
    n = sum(c.n for c in dbs)
    sig = signature(f"batch{len(dbs)}", n, max(c.m for c in dbs), sum(c.nnz for c in dbs),
                    int(sum(minsups) // max(1, len(minsups))), flags)
    hit = _cached(cache_path, sig)
    if hit:
        cfg = {k: v for k, v in hit.items() if not k.startswith("_")}
        apply(ctx, cfg)
        return cfg, hit.get("_ms"), []

    def run():
        if desc is not None:
            fim.fim_mine_batched(ctx, desc, flags=flags)
        else:
            fim.fim_mine_batched(ctx, dbs, minsups, flags)

    best, ms, table = _coordinate_search(ctx, run, space or BATCH_SPACE, BATCH_DEFAULT, repeats)
    _store(cache_path, sig, best, ms)
    return best, ms, table
