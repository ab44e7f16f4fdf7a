#!/usr/bin/env python
"""Benchmark of the GB300 Boolean-matrix frequent-itemset miner.

Default workload (the headline): 4,096 independent databases mined by the
learned+batched miner -- one graph-replayed batched pass steered by the
scheduling network, trained first on the GPU from plain-miner traces of other
databases of the same generator -- against the plain miner (one
fim_build_bitmaps + fim_mine + fim_fetch_results per database) and against the
batched pass without the network.  One step = one mine of all 4,096
databases: bit-column construction (Eq. 1), singleton and pair supports
(Eq. 2-3), the depth-first prefix extension and the canonical compaction.
`value` is itemset supports per second (support values computed: singletons
+ pairs + prefix extensions) over the device time of a step (CUDA events on
the miner's stream, CSRs resident in HBM, L2 flushed between steps); `e2e`
is the same with the CSRs uploaded from pinned host memory and every result
copied back to pinned host memory inside the timed region; `compare` holds
both times for all three arms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference      # the CPU oracle on the host cores

Single-database workloads (--workload quest_1M_1000 and the others) time one
mine per step the same way; there, --learned trains the network first, and
after the timed mines the association rules of the last one are timed once
more (--rules-ppm).  Under torchrun (N > 1) every rank mines its own replica
of the workload; the value is the supports of all ranks over the slowest
rank's time.  With --shard the ranks instead split one mine (prefix-class
shards, the parts gathered and merged on rank 0; strong scaling, also
runnable at N = 1).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "batched_4096"
HEADLINE_METRIC = "itemset supports/sec & end-to-end mine time: learned+batched vs plain, 1 GB300"
WORKLOAD_DESC = {
    "grocery_like_10k_169": "10,000 x 169, Zipf(1.0), Poisson(4.4) lengths, minsup 100",
    "quest_1M_1000": "1,000,000 x 1,000 Quest-style (T10, I4, 2,000 patterns, 50% corruption), minsup 1,000 (0.1%)",
    "planted_100k_2000": "100,000 x 2,000, Zipf(1.1) background + 500 planted patterns of length 6-12, minsup 500",
    "quest_10M_5000": "10,000,000 x 5,000 Quest-style (T12, I5, 5,000 patterns), minsup 5,000 (0.05%)",
    "batched_4096": "4,096 independent databases, n = 10^U(3,5), m ~ U{64..512}, Zipf(0.8), Poisson(6), "
                    "minsup 2% each",
}
L2_FLUSH_BYTES = 256 << 20


def _emit(line: dict) -> None:
    """Print the result line last: NCCL writes its version line through the C
    library's stdout buffer, which would otherwise be flushed after Python's."""
    import ctypes
    try:
        ctypes.CDLL(None).fflush(None)
    except (OSError, AttributeError):
        pass
    print(json.dumps(line), flush=True)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--flags", type=int, default=0, help="extra fim_mine flags")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="split one mine over the ranks (prefix-class shards, gather + merge on rank 0) "
                         "instead of one replica per rank")
    ap.add_argument("--rules-ppm", type=int, default=500_000,
                    help="also time association rules at this confidence (ppm); -1 skips")
    ap.add_argument("--n-db", type=int, default=4096,
                    help="batched workload: mine only its first N databases (profiling captures)")
    ap.add_argument("--csr", default="compact", choices=["compact", "wide"],
                    help="batched workload: the CSRs every arm reads, compact (uint32 row offsets, "
                         "uint16 item ids; FIM_CSR_COMPACT) or wide (int64, int32)")
    ap.add_argument("--learned", action="store_true",
                    help="single database: mine with FIM_LEARNED, the network trained on the GPU "
                         "from plain-miner traces of the same generator at another seed")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9
                          for i, v in enumerate(r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sm)}


def _kernel_traffic(kernel: str, workload: str):
    """ncu DRAM bytes per launch from profiles/traffic.json, if taken on the
    current source of that kernel's file; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[kernel][workload]
        src = os.path.join(ROOT, "paper_2412_19420_gb300", "csrc", e["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != e["source_sha256"]:
            return None
        return int(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _load_workload(name):
    from paper_2412_19420_gb300 import datagen
    fn, minsup = datagen.WORKLOADS[name]
    return fn(), minsup


def cpu_baseline(csr, minsup, budget_s=20.0, threads=None, frac=1.0):
    """The oracle (plain Apriori, all host cores unless `threads` is given) on
    a bounded sample of the workload: the first n' transactions, with minsup
    scaled by n'/n, starting from the fraction `frac` of the workload."""
    import numpy as np
    import oracle
    from paper_2412_19420_gb300 import datagen
    cores = threads or _cores()
    n = csr.n
    while True:
        n_s = max(1, int(n * frac))
        ms = max(1, int(round(minsup * n_s / n)))
        ip = csr.indptr[: n_s + 1]
        ix = csr.indices[: int(ip[-1])]
        t0 = time.perf_counter()
        r = oracle.apriori(ip, ix, csr.m, ms, threads=cores)
        dt = time.perf_counter() - t0
        if dt <= budget_s * 1.5 or frac <= 1 / 64:
            break
        frac /= 2 ** max(1, int(np.log2(dt / budget_s)))
    _ = datagen
    sample = ("full workload" if n_s == n else
              f"first {n_s:,} of {n:,} transactions, minsup {ms:,}") + \
        f"; {r.n_candidates:,} candidate supports counted, {len(r):,} frequent itemsets"
    return {"value": r.n_candidates / dt, "unit": "supports/s", "cores": cores, "kind": "oracle",
            "sample": sample, "seconds": round(dt, 3), "frac": n_s / max(1, n)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "batched_4096":
        run_reference_batched(args)
        return
    csr, minsup = _load_workload(args.workload)
    for _ in range(args.warmup):
        pass  # the oracle has no warm state; warm-up steps would only repeat the work
    times, vals = [], []
    for _ in range(args.steps):
        b = cpu_baseline(csr, minsup, budget_s=10.0)
        times.append(b["seconds"])
        vals.append(b["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": "itemset supports/sec", "value": value, "unit": "supports/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
            "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload]},
            "cpu_baseline": {"value": value, "unit": "supports/s", "cores": b["cores"], "kind": "oracle",
                             "sample": b["sample"]},
            "e2e": {"value": value, "unit": "supports/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _emit(line)


def _train_scheduler(ctx, fim, sched, datagen, sample):
    """The learned scheduler, trained on the GPU from plain-miner traces of a
    disjoint seeded sample of the same workload shape."""
    xs, ts = [], []
    for c, ms in sample:
        x, t = sched.collect_traces(ctx, c, ms)
        xs.append(x)
        ts.append(t)
    import numpy as np
    x, t = np.concatenate(xs), np.concatenate(ts)
    w, hist = sched.fit(ctx, x, t, steps=1500, lr=2e-3, seed=0)
    fim.fim_sched_load_weights(ctx, w)
    return {"trace_rows": int(len(x)), "final_loss": float(np.mean(hist[-50:]))}


BATCH_PPM = 20_000  # minsup 2% of each database's transactions


def _batched_workload(n_db=4096):
    """The batch's databases (the first n_db of the 4,096; fewer only for
    profiling captures), their thresholds and the line's `config` (the same
    dict on both arms: it names the workload, nothing measured)."""
    from paper_2412_19420_gb300 import datagen
    dbs = datagen.batched_dbs(datagen.batched_specs(4096)[:n_db])
    ms = [datagen.minsup_from_ppm(c.n, BATCH_PPM) for c in dbs]
    cfg = {"workload": "batched_4096", "desc": WORKLOAD_DESC["batched_4096"], "n_db": len(dbs),
           "n_trans_total": int(sum(c.n for c in dbs)), "nnz_total": int(sum(c.nnz for c in dbs)),
           "minsup_ppm": BATCH_PPM, "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)"}
    return dbs, ms, cfg


def _oracle_batch(dbs, ms, start, budget_s, threads):
    """The oracle over databases start, start+1, ... (wrapping) until budget_s
    of wall time has passed: (candidate supports, seconds, databases)."""
    import oracle
    t0 = time.perf_counter()
    cand, k = 0, 0
    while k < len(dbs) and (k == 0 or time.perf_counter() - t0 < budget_s):
        d = (start + k) % len(dbs)
        cand += oracle.apriori(dbs[d].indptr, dbs[d].indices, dbs[d].m, ms[d], threads=threads).n_candidates
        k += 1
    return cand, time.perf_counter() - t0, k


def run_reference_batched(args):
    """The oracle as the reference arm on the 4,096-database workload: each
    step mines the next databases of the batch (wrapping) for about 3 s of
    wall time on all host cores."""
    dbs, ms, cfg = _batched_workload(args.n_db)
    cores = _cores()
    times, cands, done, start = [], [], 0, 0
    for _ in range(args.steps):
        c, dt, k = _oracle_batch(dbs, ms, start, 3.0, cores)
        start = (start + k) % len(dbs)
        times.append(dt)
        cands.append(c)
        done += k
    value = sum(cands) / sum(times)
    sample = (f"{args.steps} steps of about 3 s, each the next databases of the batch in order "
              f"({done:,} database mines in all, {sum(cands):,} candidate supports counted)")
    line = {"impl": "reference", "metric": HEADLINE_METRIC, "value": value, "unit": "supports/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded generator, paper_2412_19420_gb300.datagen)",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "supports/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "supports/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _emit(line)


def _batched_roofline(st, phase, dbs, m_freq, probes, compact=False):
    """Roofline of the batch graph's dominant phase.  st: fim_get_stats of a
    timed learned+batched mine; phase: mean CUDA-event phase times (ms);
    compact: the CSRs hold uint32 row offsets and uint16 item ids."""
    hbm, _, _, src = _peaks()
    dom = max(("ms_build", "ms_pairs", "ms_dfs", "ms_compact"), key=lambda p: phase[p])
    sec = phase[dom] / 1000
    if dom == "ms_build":
        # CSR read once, bit columns written once, the singleton supports fused
        po, pi = (4, 2) if compact else (8, 4)
        nbytes = sum(po * (c.n + 1) + pi * c.nnz + 4 * c.m * ((c.n + 31) // 32) for c in dbs)
        ach = nbytes / sec / 1e9
        roof = {"kernel": "batch_build_rows_kernel", "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": _kernel_traffic("batch_build_rows_kernel", "batched_4096"),
                "algorithmic_bytes_per_launch": int(nbytes)}
    elif dom == "ms_pairs":
        # AND + popc of every word pair of the frequent items' columns
        wp = sum(mf * (mf - 1) // 2 * ((c.n + 31) // 32) for c, mf in zip(dbs, m_freq))
        ach = wp / sec
        peak = probes["popc_word_pairs_per_s"]
        if st["pair_path"] == 1:
            # tensor cores: the pair supports' flops (2 per word-pair bit) against
            # the measured f8f6f4 rate at the tiles' width (A from shared memory)
            fl = 64.0 * wp
            peak_t = probes.get("mma_f8f6f4_tflops_n128") or probes["mma_f8f6f4_tflops_a_smem"]
            roof = {"kernel": "batch_pairs_tc_kernel", "bound": "tensor", "achieved": fl / sec / 1e12,
                    "peak": peak_t, "unit": "TFLOP/s", "frac": fl / sec / 1e12 / peak_t,
                    "traffic": _kernel_traffic("batch_pairs_tc_kernel", "batched_4096"),
                    "peak_source": "measured tcgen05 f8f6f4 rate at N = 128 (fim_probe 4)",
                    "algorithmic_word_pairs_per_launch": int(wp)}
        else:
            roof = {"kernel": "batch_pairs_kernel", "bound": "alu", "achieved": ach / 1e9, "peak": peak / 1e9,
                    "unit": "Gwordpairs/s", "frac": ach / peak, "traffic": None, "peak_source": "fim_probe AND/popc",
                    "algorithmic_word_pairs_per_launch": int(wp)}
    elif dom == "ms_dfs":
        # warp workers (eight per CTA) when the batch's columns are short
        kern = "dfs_warp_kernel" if st["dfs_workers"] > 1024 else "dfs_kernel"
        roof = _dfs_roofline(st, phase[dom], "batched_4096", probes, kern)
    else:
        nbytes = 24 * st["n_sets"]
        ach = nbytes / sec / 1e9
        roof = {"kernel": "compaction", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": None}
    roof.setdefault("peak_source", src)
    roof["phase_ms"] = {k: round(v, 4) for k, v in phase.items()}
    return roof


def run_batched(args):
    """4,096 independent databases, the metric's comparison on one GPU: the
    learned+batched miner (one graph-replayed batched pass, FIM_LEARNED)
    against the plain miner (one fim_build_bitmaps + fim_mine +
    fim_fetch_results per database) and against the batched pass without the
    network.  Each arm is timed on the device (CSRs resident in HBM, results
    left canonical on the device) and end to end (CSRs uploaded from pinned
    host memory and every result copied back to pinned host memory inside
    the timed region)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2412_19420_gb300 import datagen, fim, sched

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    dbs, ms, cfg = _batched_workload(args.n_db)
    compact = args.csr == "compact"
    cfg = dict(cfg, csr=("compact: uint32 row offsets, uint16 item ids (FIM_CSR_COMPACT), every arm"
                         if compact else "wide: int64 row offsets, int32 item ids, every arm"))
    # the arrays every arm reads: the generator's CSR, or the same rows with
    # narrower element types (bit patterns kept in the signed torch dtypes)
    ptr_dt, idx_dt = (np.uint32, np.uint16) if compact else (np.int64, np.int32)
    stream = torch.cuda.Stream()
    ctx = fim.fim_create(local, stream)
    # the network: trained on the GPU from plain-miner traces of 48 other
    # databases of the same generator (seed 1)
    train_sample = [datagen.batched_db(s) for s in datagen.batched_specs(48, seed=1)]
    train_sample = [(c, datagen.minsup_from_ppm(c.n, BATCH_PPM)) for c in train_sample]
    train_info = _train_scheduler(ctx, fim, sched, datagen, train_sample)

    t_ptr, t_idx = (np.int32, np.int16) if compact else (np.int64, np.int32)

    class Dev:
        def __init__(self, c):
            ix = c.indices if c.nnz else np.zeros(1, np.int32)
            self.indptr = torch.from_numpy(c.indptr.astype(ptr_dt).view(t_ptr)).cuda()
            self.indices = torch.from_numpy(ix.astype(idx_dt).view(t_idx)).cuda()
            self.m = c.m
    ddbs = [Dev(c) for c in dbs]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def timed(fn, reps, host_clock=False):
        """Per-rep ms: CUDA events on the miner's stream (device arms) or the
        host clock around a call that ends synchronised (end-to-end arms)."""
        out = []
        for k in range(reps):
            with torch.cuda.stream(stream):
                flush.fill_(k)
            if host_clock:
                stream.synchronize()
                t0 = time.perf_counter()
                fn()
                stream.synchronize()
                out.append(1000 * (time.perf_counter() - t0))
                continue
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    learned = fim.FIM_LEARNED | args.flags
    plain_flags = args.flags
    # ---- learned + batched, device-resident inputs: the line's value -------
    # (the descriptor table is marshalled once, as a C caller holds its
    # fim_db_desc array); launch shapes picked by the autotuner first
    ddesc = fim.BatchDescriptor(ddbs, ms)
    from paper_2412_19420_gb300 import autotune
    tuned, tuned_ms, tune_table = autotune.tune_batched(ctx, dbs, ms, flags=learned, desc=ddesc)
    cfg = dict(cfg, tuned={k: int(tuned[k]) for k in sorted(autotune.BATCH_SPACE)})
    for _ in range(args.warmup):
        fim.fim_mine_batched(ctx, ddesc, flags=learned)
    barrier()
    phase = {k: 0.0 for k in ("ms_build", "ms_pairs", "ms_dfs", "ms_compact")}
    launches = 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k)
            ev[k][0].record(stream)
            fim.fim_mine_batched(ctx, ddesc, flags=learned)
            ev[k][1].record(stream)
            st = fim.fim_get_stats(ctx)
            for p in phase:
                phase[p] += st[p]
            launches += st["launches_mine"]
        barrier()
    lb = [a.elapsed_time(b) for a, b in ev]
    phase = {p: v / args.steps for p, v in phase.items()}
    st = fim.fim_get_stats(ctx)
    supports = st["supports_singletons"] + st["supports_pairs"] + st["supports_dfs"]
    R, T = fim.fim_batch_sizes(ctx, fim.FIM_ALL_DBS)
    ms_lb = statistics.mean(lb)
    t = torch.tensor([ms_lb], dtype=torch.float64, device="cuda")
    tot = torch.tensor([float(supports)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    value = float(tot.item()) / (ms_max / 1000)

    # ---- the other device arms --------------------------------------------
    batched_plain = timed(lambda: fim.fim_mine_batched(ctx, ddesc, flags=plain_flags), max(3, args.steps // 2))
    out_d = (torch.empty(1 << 20, dtype=torch.int64, device="cuda"),
             torch.empty(1 << 22, dtype=torch.int32, device="cuda"),
             torch.empty(1 << 20, dtype=torch.int32, device="cuda"))

    # the plain miner runs with the library's default launch shapes
    batched_shape = {k: tuned[k] for k in tuned}
    autotune.apply(ctx, autotune.DEFAULT)

    def plain_device():
        for c, m in zip(ddbs, ms):
            fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
            fim.fim_mine(ctx, m, plain_flags)
            fim.fim_fetch_results(ctx, out_d)
    plain_device()
    plain = timed(plain_device, 2)

    # ---- end to end: host CSRs in, every result back in pinned host memory
    out_h = (torch.empty(R + 1, dtype=torch.int64).pin_memory(), torch.empty(max(T, 1), dtype=torch.int32).pin_memory(),
             torch.empty(max(R, 1), dtype=torch.int32).pin_memory())
    out_hn = tuple(x.numpy() for x in out_h)
    # the CSRs in pinned host memory, packed back to back (the library uploads
    # contiguous databases in one copy per array)
    n_ptr = sum(c.n + 1 for c in dbs)
    n_idx = sum(c.nnz for c in dbs)
    ptr_h = torch.empty(n_ptr, dtype=torch.int32 if compact else torch.int64).pin_memory().numpy().view(ptr_dt)
    idx_h = torch.empty(max(n_idx, 1), dtype=torch.int16 if compact else torch.int32).pin_memory().numpy().view(idx_dt)
    hdbs, po, io = [], 0, 0
    for c in dbs:
        ptr_h[po:po + c.n + 1] = c.indptr
        idx_h[io:io + c.nnz] = c.indices
        hdbs.append(datagen.Csr(indptr=ptr_h[po:po + c.n + 1], indices=idx_h[io:io + c.nnz], m=c.m))
        po += c.n + 1
        io += c.nnz
    hdesc = fim.BatchDescriptor(hdbs, ms)

    def e2e_batched(flags):
        autotune.apply(ctx, batched_shape)
        fim.fim_mine_batched(ctx, hdesc, flags=flags)
        fim.fim_fetch_batched(ctx, fim.FIM_ALL_DBS, out_hn)

    def plain_host():
        autotune.apply(ctx, autotune.DEFAULT)
        for c, m in zip(hdbs, ms):
            fim.fim_build_bitmaps(ctx, c.indptr, c.indices, c.m)
            fim.fim_mine(ctx, m, plain_flags)
            fim.fim_fetch_results(ctx, out_hn)
    for _ in range(max(1, args.warmup)):
        e2e_batched(learned)
    e2e_lb = timed(lambda: e2e_batched(learned), args.steps, host_clock=True)
    e2e_bp = timed(lambda: e2e_batched(plain_flags), max(3, args.steps // 2), host_clock=True)
    plain_host()
    e2e_plain = timed(plain_host, 2, host_clock=True)
    e2e_t = torch.tensor([statistics.mean(e2e_lb)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    h2d = sum(c.indptr.nbytes + c.indices.nbytes for c in hdbs)
    d2h = 8 * (R + 1) + 4 * T + 4 * R

    # frequent items per database (the sets of size 1 of each slice)
    autotune.apply(ctx, batched_shape)
    fim.fim_mine_batched(ctx, hdesc, flags=learned)
    res = fim.fim_fetch_batched(ctx, fim.FIM_ALL_DBS, out_hn)
    sl = fim.fim_batch_slices(ctx, len(dbs)).astype(np.int64)
    single = (np.diff(res.offsets.astype(np.int64)) == 1).astype(np.int64)
    csum = np.concatenate([[0], np.cumsum(single)])
    m_freq = [int(csum[sl[d + 1]] - csum[sl[d]]) for d in range(len(dbs))]

    probes = _probes(fim, ctx)
    roof = _batched_roofline(st, phase, dbs, m_freq, probes, compact)
    med = statistics.median
    compare = {
        "unit": f"ms per mine of all {len(dbs):,} databases",
        "device": {"learned_batched": ms_lb, "batched_plain": med(batched_plain), "plain_per_database": med(plain)},
        "e2e": {"learned_batched": statistics.mean(e2e_lb), "batched_plain": med(e2e_bp),
                "plain_per_database": med(e2e_plain)},
        "speedup_learned_batched_vs_plain": {"device": med(plain) / ms_lb,
                                             "e2e": med(e2e_plain) / statistics.mean(e2e_lb)},
        "network_gain_vs_batched_plain": {"device": med(batched_plain) / ms_lb,
                                          "e2e": med(e2e_bp) / statistics.mean(e2e_lb)},
        "timing": "device: CUDA events on the miner's stream; e2e: host clock around calls that end "
                  "synchronised; L2 flushed before every rep",
    }
    line = {
        "metric": HEADLINE_METRIC, "value": value, "unit": "supports/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generator, paper_2412_19420_gb300.datagen)",
        "config": cfg,
        "e2e": {"value": float(tot.item()) / (float(e2e_t.item()) / 1000), "unit": "supports/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(e2e_t.item())},
        "compare": compare,
        "gpu_launches": int(launches),
        "roofline": roof,
        "probes": probes,
        "details": {"mode": "learned+batched (FIM_LEARNED, one graph-replayed batched pass)",
                    "parallelism": f"replicas x{world}" if world > 1 else "one GPU",
                    "frequent_itemsets": int(R), "max_len": int(st["max_len"]),
                    "supports_per_step": int(supports), "classes": int(st["classes"]),
                    "diffset_classes": int(st["diffset_classes"]),
                    "dfs_utilisation": (st["dfs_busy_ns"] / max(1, st["dfs_span_ns"] * st["dfs_workers"])),
                    "peak_device_mib": round(st["peak_device_bytes"] / 2**20, 1),
                    "scheduler_training": train_info,
                    "autotune": {"ms_best": tuned_ms, "tried": [[{k: c[k] for k in sorted(autotune.BATCH_SPACE)},
                                                                 round(t, 4)] for c, t in tune_table]}},
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cand, dt, k = _oracle_batch(dbs, ms, 0, 25.0, _cores())
        line["cpu_baseline"] = {"value": cand / dt, "unit": "supports/s", "cores": _cores(), "kind": "oracle",
                                "sample": (f"{'all' if k == len(dbs) else f'the first {k} of'} {len(dbs)} databases "
                                           f"({cand:,} candidate supports), {dt:.1f} s")}
    if rank == 0:
        _emit(line)
    fim.fim_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args):
    """One mine of the workload split over the ranks: every rank builds the
    whole matrix and mines its prefix-class shard (fim_mine_shard), the parts
    are gathered on rank 0 (torch.distributed over NCCL) and merged into the
    canonical answer (fim_merge_results), which rank 0 fetches.  Strong
    scaling: the job's work is one mine whatever the rank count."""
    import socket

    import torch
    import torch.distributed as dist
    from paper_2412_19420_gb300 import fim, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    else:  # the gather still runs, over a one-rank group
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    csr, minsup = _load_workload(args.workload)
    stream = torch.cuda.Stream()
    ctx = fim.fim_create(local, stream)
    flags = args.flags
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def mine(ip, ix, out_final):
        """One step; returns (stats of this rank's shard mine, merge stats or None)."""
        fim.fim_build_bitmaps(ctx, ip, ix, csr.m)
        fim.fim_mine_shard(ctx, minsup, flags, rank, world)
        st_mine = fim.fim_get_stats(ctx)
        R, T = fim.fim_result_sizes(ctx)
        part = (torch.empty(R + 1, dtype=torch.int64, device="cuda"),
                torch.empty(max(T, 1), dtype=torch.int32, device="cuda"),
                torch.empty(max(R, 1), dtype=torch.int32, device="cuda"))
        fim.fim_fetch_results(ctx, part)
        parts = shard.gather_parts((part[0], part[1][:T], part[2][:R]))
        if rank != 0:
            torch.cuda.current_stream().synchronize()  # the sends have left
            return st_mine, None
        fim.fim_merge_results(ctx, csr.n, csr.m, parts)
        st_merge = fim.fim_get_stats(ctx)
        fim.fim_fetch_results(ctx, out_final)
        return st_mine, st_merge

    ip_d = torch.from_numpy(csr.indptr).cuda()
    ix_d = torch.from_numpy(csr.indices).cuda()
    fim.fim_build_bitmaps(ctx, ip_d, ix_d, csr.m)
    fim.fim_mine(ctx, minsup, flags)
    R, T = fim.fim_result_sizes(ctx)  # the merged answer's size
    out_d = (torch.empty(R + 1, dtype=torch.int64, device="cuda"),
             torch.empty(max(T, 1), dtype=torch.int32, device="cuda"),
             torch.empty(max(R, 1), dtype=torch.int32, device="cuda"))
    for _ in range(args.warmup):
        mine(ip_d, ix_d, out_d)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase = {k: 0.0 for k in ("ms_build", "ms_singletons", "ms_pairs", "ms_dfs", "ms_compact")}
    launches, merge_ms = 0, 0.0
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k)
            ev[k][0].record(stream)
            st_mine, st_merge = mine(ip_d, ix_d, out_d)
            ev[k][1].record(stream)
            for p in phase:
                phase[p] += st_mine[p]
            launches += st_mine["launches_build"] + st_mine["launches_mine"]
            if st_merge is not None:
                launches += st_merge["launches_mine"]
                merge_ms += st_merge["ms_compact"]
        barrier()
    ms_step = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # the job's supports: singletons and pairs once (every rank computes them),
    # the DFS supports of every shard
    t = torch.tensor([ms_step], dtype=torch.float64, device="cuda")
    dfs = torch.tensor([float(st_mine["supports_dfs"])], dtype=torch.float64, device="cuda")
    lc = torch.tensor([float(launches)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(dfs, op=dist.ReduceOp.SUM)
    dist.all_reduce(lc, op=dist.ReduceOp.SUM)
    supports = st_mine["supports_singletons"] + st_mine["supports_pairs"] + dfs.item()
    ms_max = float(t.item())
    value = supports / (ms_max / 1000.0)

    # e2e: host CSR on every rank, the merged answer to pinned host memory on rank 0
    ip_h = torch.from_numpy(csr.indptr).pin_memory()
    ix_h = torch.from_numpy(csr.indices).pin_memory()
    out_h = tuple(torch.empty(x.shape[0], dtype=x.dtype).pin_memory() for x in out_d)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k)
        barrier()
        t0 = time.perf_counter()
        mine(ip_h.numpy(), ix_h.numpy(), tuple(x.numpy() for x in out_h))
        if k >= args.warmup:
            e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_t = torch.tensor([statistics.mean(e2e_ms)], dtype=torch.float64, device="cuda")
    dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = supports / (float(e2e_t.item()) / 1000.0)

    avg = {p: phase[p] / args.steps for p in phase}
    roof = _roofline(st_mine, avg, csr, args.workload, _probes(fim, ctx))
    line = {
        "metric": "itemset supports/sec", "value": value, "unit": "supports/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generator, paper_2412_19420_gb300.datagen)",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload],
                   "n_trans": csr.n, "n_items": csr.m, "minsup": minsup, "flags": flags,
                   "parallelism": f"prefix-class shards x{world}, gather + merge on rank 0",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "frequent_itemsets": int(R), "merge_ms": round(merge_ms / args.steps, 4),
                   "supports_per_step": int(supports)},
        "e2e": {"value": e2e_value, "unit": "supports/s",
                "h2d_bytes_per_step": int(world * (csr.indptr.nbytes + csr.indices.nbytes)),
                "d2h_bytes_per_step": int(8 * (R + 1) + 4 * T + 4 * R), "ms_per_step": float(e2e_t.item())},
        "gpu_launches": int(lc.item()),
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if rank == 0:
        _emit(line)
    fim.fim_destroy(ctx)
    dist.destroy_process_group()


def _probes(fim, ctx):
    """Measured ceilings on this GPU: the AND/popc word-pair rate, the L2 read
    bandwidth (the L2-resident operands' ceiling) and the tcgen05 f8f6f4 MMA
    rate with A from tensor or shared memory."""
    return {"popc_word_pairs_per_s": fim.fim_probe(ctx, 0), "l2_read_gbs": fim.fim_probe(ctx, 1),
            "mma_f8f6f4_tflops_a_tmem": fim.fim_probe(ctx, 2), "mma_f8f6f4_tflops_a_smem": fim.fim_probe(ctx, 3),
            "mma_f8f6f4_tflops_n128": fim.fim_probe(ctx, 4), "mma_f8f6f4_tflops_n64": fim.fim_probe(ctx, 5)}


def _dfs_roofline(st, ms_dfs, workload, probes, kernel="dfs_kernel"):
    """The prefix-extension kernel against its ceiling.  Its algorithmic bytes
    are those of the operands the chosen representations stream, at 32-byte
    sector granularity (zero sectors skipped, sparse classes as (index,
    word) pairs); the dense-column figure is reported beside it.  Where the
    ncu DRAM traffic of the kernel (taken on its current source) is well
    below those bytes, they are served by L2, and the ceiling is the measured
    L2 read bandwidth; else HBM.  Both fractions are reported either way."""
    hbm, _, _, src = _peaks()
    sec = ms_dfs / 1000
    ach = st["dfs_touched_bytes"] / sec / 1e9
    traffic = _kernel_traffic(kernel, workload)
    l2 = probes["l2_read_gbs"]
    roof = {"kernel": kernel, "achieved": ach, "unit": "GB/s", "traffic": traffic,
            "algorithmic_bytes_per_launch": st["dfs_touched_bytes"],
            "dense_equivalent_bytes_per_launch": st["dfs_bytes"],
            "hbm_frac": ach / hbm, "l2_frac": ach / l2,
            "alu_frac": st["dfs_touched_bytes"] / 4 / sec / probes["popc_word_pairs_per_s"]}
    if traffic is not None:
        roof["dram_frac"] = traffic / sec / 1e9 / hbm
    if traffic is not None and traffic < 0.5 * st["dfs_touched_bytes"]:
        roof.update({"bound": "l2", "peak": l2, "frac": ach / l2, "peak_source": "measured L2 read (fim_probe 1)"})
    else:
        roof.update({"bound": "hbm", "peak": hbm, "frac": ach / hbm, "peak_source": src})
    return roof


def _roofline(st, avg, csr, workload, probes):
    """Roofline of the dominant phase of a mine: st = fim_get_stats of a
    timed mine, avg = mean CUDA-event phase times (ms); probes = fim_probe's
    measured AND/popc rate, L2 bandwidth and tcgen05 f8f6f4 rate (the pair
    pass's ceiling)."""
    mma_tflops = probes.get("mma_f8f6f4_tflops_a_tmem")
    hbm, bf16, bf16_s, src = _peaks()
    dom = max(("ms_pairs", "ms_dfs", "ms_compact", "ms_build"), key=lambda p: avg[p])
    if dom == "ms_dfs":
        roof = _dfs_roofline(st, avg[dom], workload, probes)
    elif dom == "ms_pairs" and st["pair_path"] == 1:
        fl = 2.0 * st["supports_pairs"] * csr.n
        ach = fl / (avg[dom] / 1000) / 1e12
        if mma_tflops:
            peak, psrc = mma_tflops, "measured tcgen05 f8f6f4 rate (fim_probe 2)"
        else:
            peak, psrc = 2 * bf16, f"2 x {src} bf16 (nominal fp8 / bf16 ratio)"
        roof = {"kernel": "pairs_tc_kernel", "bound": "tensor", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "peak_source": psrc,
                "traffic": _kernel_traffic("pairs_tc_kernel", workload)}
    else:
        nm = {"ms_pairs": "pairs_popc_kernel", "ms_compact": "compaction", "ms_build": "build_bitmaps_kernel"}[dom]
        nbytes = {"ms_pairs": 4 * st["n_frequent_items"] * ((csr.n + 31) // 32),
                  "ms_compact": 24 * st["n_sets"],
                  "ms_build": csr.indptr.nbytes + csr.indices.nbytes + 4 * csr.m * ((csr.n + 31) // 32)}[dom]
        ach = nbytes / (avg[dom] / 1000) / 1e9
        roof = {"kernel": nm, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": _kernel_traffic(nm, workload)}
    roof.setdefault("peak_source", src)
    roof["phase_ms"] = {k: round(v, 4) for k, v in avg.items()}
    return roof


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched_4096":
        run_batched(args)
        return
    if args.shard:
        run_sharded(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2412_19420_gb300 import fim

    csr, minsup = _load_workload(args.workload)
    stream = torch.cuda.Stream()
    ctx = fim.fim_create(local, stream)
    training = None
    if args.learned:
        from paper_2412_19420_gb300 import datagen, sched
        fn, _ = datagen.WORKLOADS[args.workload]
        training = _train_scheduler(ctx, fim, sched, datagen, [(fn(seed=1), minsup)])
    ip_d = torch.from_numpy(csr.indptr).cuda()
    ix_d = torch.from_numpy(csr.indices).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    flags = args.flags | (fim.FIM_LEARNED if args.learned else 0)

    def mine_device(out):
        fim.fim_build_bitmaps(ctx, ip_d, ix_d, csr.m)
        fim.fim_mine(ctx, minsup, flags)
        return fim.fim_fetch_results(ctx, out)

    # size the device output buffers once
    fim.fim_build_bitmaps(ctx, ip_d, ix_d, csr.m)
    fim.fim_mine(ctx, minsup, flags)
    R, T = fim.fim_result_sizes(ctx)
    out_d = (torch.empty(R + 1, dtype=torch.int64, device="cuda"),
             torch.empty(max(T, 1), dtype=torch.int32, device="cuda"),
             torch.empty(max(R, 1), dtype=torch.int32, device="cuda"))
    for _ in range(args.warmup):
        mine_device(out_d)
    barrier()

    # ---- timed: device-resident input, results left on the device -------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase = {k: 0.0 for k in ("ms_build", "ms_singletons", "ms_pairs", "ms_dfs", "ms_compact")}
    launches = 0
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k)
            ev[k][0].record(stream)
            mine_device(out_d)
            ev[k][1].record(stream)
            st = fim.fim_get_stats(ctx)
            for p in phase:
                phase[p] += st[p]
            launches += st["launches_build"] + st["launches_mine"]
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = sum(step_ms) / len(step_ms)
    st = fim.fim_get_stats(ctx)
    supports = st["supports_singletons"] + st["supports_pairs"] + st["supports_dfs"]
    t = torch.tensor([ms_step], dtype=torch.float64, device="cuda")
    tot = torch.tensor([float(supports)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    value = float(tot.item()) / (ms_max / 1000.0)

    # ---- e2e: host CSR in, host results out, copies inside the timed region
    ip_h = torch.from_numpy(csr.indptr).pin_memory()
    ix_h = torch.from_numpy(csr.indices).pin_memory()
    out_h = (torch.empty(R + 1, dtype=torch.int64).pin_memory(),
             torch.empty(max(T, 1), dtype=torch.int32).pin_memory(),
             torch.empty(max(R, 1), dtype=torch.int32).pin_memory())
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k)
        stream.synchronize()
        t0 = time.perf_counter()
        fim.fim_build_bitmaps(ctx, ip_h.numpy(), ix_h.numpy(), csr.m)
        fim.fim_mine(ctx, minsup, flags)
        got = fim.fim_fetch_results(ctx, tuple(x.numpy() for x in out_h))
        if k >= args.warmup:
            e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_t = torch.tensor([statistics.mean(e2e_ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = float(tot.item()) / (float(e2e_t.item()) / 1000.0)
    h2d = csr.indptr.nbytes + csr.indices.nbytes
    d2h = 8 * (R + 1) + 4 * T + 4 * R

    # ---- association rules of the last mine (a post-pass, not in the step)
    rules = None
    if args.rules_ppm >= 0:
        fim.fim_rules(ctx, args.rules_ppm)  # sizes the rule buffers
        rule_ms = []
        for _ in range(max(3, args.steps)):
            stream.synchronize()
            t0 = time.perf_counter()
            n_rules = fim.fim_rules(ctx, args.rules_ppm)
            rule_ms.append(1000 * (time.perf_counter() - t0))
        evaluated = fim.fim_rules_evaluated(ctx)
        ms_r = statistics.median(rule_ms)
        rules = {"min_conf_ppm": args.rules_ppm, "n_rules": int(n_rules), "antecedents_evaluated": evaluated,
                 "ms": round(ms_r, 4), "rules_per_s": n_rules / (ms_r / 1000),
                 "antecedents_per_s": evaluated / (ms_r / 1000),
                 "timing": "host wall clock around fim_rules (keep and write passes, two scans, "
                           "three host syncs), median"}

    # ---- roofline of the dominant phase ---------------------------------
    avg = {p: phase[p] / args.steps for p in phase}
    probes = _probes(fim, ctx)
    roof = _roofline(st, avg, csr, args.workload, probes)

    from paper_2412_19420_gb300 import report
    tables = report.table_columns(out_d[2][:R], csr.n, st)
    line = {
        "metric": "itemset supports/sec", "value": value, "unit": "supports/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generator, paper_2412_19420_gb300.datagen)",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload],
                   "n_trans": csr.n, "n_items": csr.m, "minsup": minsup, "flags": flags,
                   "scheduler_training": training,
                   "parallelism": f"replicas x{world}",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "frequent_itemsets": int(st["n_sets"]), "max_len": int(st["max_len"]),
                   # the paper's Table 1 / Table 2 columns, on this workload
                   "avg_support_pct": round(tables["avg_support_pct"], 4),
                   "peak_device_mib": round(tables["peak_device_mib"], 1),
                   "supports_per_step": int(supports),
                   "pair_path": "tcgen05" if st["pair_path"] == 1 else "popc"},
        "e2e": {"value": e2e_value, "unit": "supports/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": float(e2e_t.item())},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk.summary(),
    }
    line["probes"] = probes
    if rules is not None:
        line["rules"] = rules
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(csr, minsup)
        # one thread: start from the sample the all-core run's time suggests
        nt = line["cpu_baseline"]
        guess = nt.pop("frac") * min(1.0, 8.0 / max(1e-3, nt["seconds"] * nt["cores"]))
        one = cpu_baseline(csr, minsup, budget_s=8.0, threads=1, frac=max(guess, 1 / 64))
        one.pop("frac")
        line["cpu_baseline"]["single_thread"] = {k: one[k] for k in ("value", "sample", "seconds")}
    if rank == 0:
        _emit(line)
    _ = (np, got)
    fim.fim_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
