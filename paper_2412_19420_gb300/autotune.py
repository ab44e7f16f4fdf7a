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
                 cache_path: str | None = None):
    """Best knob setting for a batch (DFS workers and split depth)."""
    n = sum(c.n for c in dbs)
    sig = signature(f"batch{len(dbs)}", n, max(c.m for c in dbs), sum(c.nnz for c in dbs),
                    int(sum(minsups) // max(1, len(minsups))), flags)
    hit = _cached(cache_path, sig)
    if hit:
        cfg = {k: v for k, v in hit.items() if not k.startswith("_")}
        apply(ctx, cfg)
        return cfg

    def run():
        fim.fim_mine_batched(ctx, dbs, minsups, flags)

    sp = space or {k: v for k, v in SPACE.items() if k != "pairs_kdrain"}
    best, ms, _ = _search(ctx, run, sp, repeats)
    _store(cache_path, sig, best, ms)
    return best
