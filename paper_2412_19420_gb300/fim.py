"""Python binding of libfim (include/fim.h): the same entry points, marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers and status codes to exceptions.  If libfim.so
has not been built, importing the binding raises -- there is no fallback.

    ctx = fim_create(device=0)
    fim_build_bitmaps(ctx, indptr, indices, n_items)        # numpy (host) or torch CUDA
    fim_mine(ctx, minsup)
    res = fim_fetch_results(ctx)                            # Itemsets (numpy, canonical)
    fim_destroy(ctx)
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os

import numpy as np

from . import build as _build

FIM_OK = 0
FIM_E_INVAL, FIM_E_NOMEM, FIM_E_CUDA, FIM_E_TIMEOUT = -1, -2, -3, -4
FIM_E_STACK, FIM_E_TOO_SMALL, FIM_E_STATE, FIM_E_NODEV = -5, -6, -7, -8
FIM_E_CHECK = -9
FIM_INPUT_HOST, FIM_INPUT_DEVICE = 0, 0x100
FIM_CSR_COMPACT = 0x400
FIM_OUTPUT_HOST, FIM_OUTPUT_DEVICE = 0, 0x200
FIM_STRICT, FIM_LEARNED, FIM_PAIRS_POPC, FIM_TRACE = 0x1, 0x2, 0x4, 0x8
FIM_DIFFSET_RULE, FIM_NO_SPLIT = 0x10, 0x20
FIM_MLP_PARAMS = 4866


def FIM_MAXLEN(k: int) -> int:
    return (int(k) & 0xFF) << 24


class FimError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {fim_strerror(code)} ({code})")
        self.code = code


class fim_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "n_trans", "n_items", "n_frequent_items", "n_sets", "max_len",
        "supports_singletons", "supports_pairs", "supports_dfs", "dfs_words", "dfs_bytes", "dfs_touched_bytes",
        "classes", "tasks_pushed", "diffset_classes", "peak_device_bytes",
        "launches_build", "launches_mine", "dfs_busy_ns", "dfs_span_ns", "dfs_workers", "dfs_root_ns")] + \
        [(n, ctypes.c_float) for n in ("ms_build", "ms_singletons", "ms_pairs", "ms_dfs", "ms_compact")] + \
        [("pair_path", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class fim_db_desc(ctypes.Structure):
    _fields_ = [("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("n_trans", ctypes.c_int64), ("n_items", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("minsup", ctypes.c_uint64)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libfim.so is not built ({path}); run "
                          "`python -m paper_2412_19420_gb300.build` or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, U64, I64, I32, U32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    sig = {
        "fim_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
        "fim_destroy": (None, [P]),
        "fim_build_bitmaps": (ctypes.c_int, [P, P, P, I64, I32, U32]),
        "fim_mine": (ctypes.c_int, [P, U64, U32]),
        "fim_fetch_results": (ctypes.c_int, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), P, P, P, U64, U64, U32]),
        "fim_get_stats": (ctypes.c_int, [P, ctypes.POINTER(fim_stats)]),
        "fim_mine_batched": (ctypes.c_int, [P, ctypes.c_int, P, U32]),
        "fim_fetch_batched": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(U64), ctypes.POINTER(U64),
                                             P, P, P, U64, U64, U32]),
        "fim_sched_load_weights": (ctypes.c_int, [P, P, ctypes.c_size_t]),
        "fim_fetch_traces": (ctypes.c_int, [P, ctypes.POINTER(U64), P, P, U64]),
        "fim_mlp_forward": (ctypes.c_int, [P, P, P, I64, P, P, ctypes.c_int]),
        "fim_mlp_backward": (ctypes.c_int, [P, P, P, P, P, P, I64, P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
        "fim_mlp_adam": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_float]),
        "fim_set_tuning": (ctypes.c_int, [P, ctypes.c_char_p, I64]),
        "fim_rules": (ctypes.c_int, [P, U32, ctypes.c_int, ctypes.POINTER(U64)]),
        "fim_mine_shard": (ctypes.c_int, [P, U64, U32, ctypes.c_int, ctypes.c_int]),
        "fim_merge_results": (ctypes.c_int, [P, I64, I32, ctypes.c_int, P, P, P, P, P, U32]),
        "fim_fetch_rules": (ctypes.c_int, [P, ctypes.POINTER(U64), P, P, P, P, U64, U32]),
        "fim_rules_evaluated": (ctypes.c_int, [P, ctypes.POINTER(U64)]),
        "fim_probe": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "fim_batch_slices": (ctypes.c_int, [P, P, U64]),
        "fim_pair_supports_noalloc": (ctypes.c_int, [P, P, I64, I32, P, P]),
        "fim_minsup_from_ppm": (U64, [I64, U32]),
        "fim_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "fim_version": (U32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(code: int, what: str) -> None:
    if code != FIM_OK:
        raise FimError(code, what)


def fim_strerror(code: int) -> str:
    return _lib.fim_strerror(int(code)).decode()


def fim_version() -> int:
    return int(_lib.fim_version())


def fim_minsup_from_ppm(n_trans: int, ppm: int) -> int:
    return int(_lib.fim_minsup_from_ppm(int(n_trans), int(ppm)))


def _sync_torch(*arrays) -> None:
    """Work that produced (or still uses) these CUDA tensors may be queued on
    torch's current stream; the library's stream does not wait for other
    streams, so that work is finished first."""
    for a in arrays:
        if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
            return


def _itemsize(a) -> int:
    return int(a.element_size()) if hasattr(a, "element_size") else int(a.itemsize)


def _csr_format(indptr, indices) -> int:
    """FIM_CSR_COMPACT for 4-byte row offsets with 2-byte item ids (uint32 /
    uint16, or torch int32 / int16 holding those bits), 0 for the wide int64 /
    int32 CSR; any other pairing is rejected."""
    sp, si = _itemsize(indptr), _itemsize(indices)
    if (sp, si) == (8, 4):
        return 0
    if (sp, si) == (4, 2):
        return FIM_CSR_COMPACT
    raise ValueError(f"CSR element sizes ({sp}, {si}) are neither (8, 4) nor (4, 2)")


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a.is_cuda
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, False


def fim_create(device: int = 0, stream=None):
    """New context on `device`; `stream` is a torch.cuda.Stream, an int handle or None."""
    h = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(_lib.fim_create(ctypes.byref(h), int(device), s), "fim_create")
    return h


def fim_destroy(ctx) -> None:
    _lib.fim_destroy(ctx)


def fim_build_bitmaps(ctx, indptr, indices, n_items: int, flags: int | None = None) -> None:
    """CSR -> the ctx's bit columns (Eq. 1).  Wide (int64 indptr, int32
    indices) or compact (uint32 indptr, uint16 indices: FIM_CSR_COMPACT, set
    from the arrays' element sizes)."""
    if not hasattr(indptr, "data_ptr"):
        indptr = np.asarray(indptr)
        indices = np.asarray(indices)
        if (indptr.dtype, indices.dtype) != (np.dtype(np.uint32), np.dtype(np.uint16)):
            indptr = np.ascontiguousarray(indptr, dtype=np.int64)
            indices = np.ascontiguousarray(indices, dtype=np.int32)
        else:
            indptr, indices = np.ascontiguousarray(indptr), np.ascontiguousarray(indices)
    _sync_torch(indptr, indices)
    p, dev = _ptr(indptr)
    q, dev2 = _ptr(indices)
    if dev != dev2:
        raise ValueError("indptr and indices must both be host or both be device")
    if flags is None:
        flags = FIM_INPUT_DEVICE if dev else FIM_INPUT_HOST
    flags = int(flags) | _csr_format(indptr, indices)
    n = int(indptr.shape[0]) - 1
    _check(_lib.fim_build_bitmaps(ctx, p, q, n, int(n_items), int(flags)), "fim_build_bitmaps")


def fim_mine(ctx, minsup: int, flags: int = 0) -> None:
    _check(_lib.fim_mine(ctx, int(minsup), int(flags)), "fim_mine")


@dataclasses.dataclass
class Itemsets:
    offsets: np.ndarray   # uint64[R+1]
    items: np.ndarray     # uint32
    supports: np.ndarray  # uint32[R]

    def __len__(self) -> int:
        return int(self.supports.shape[0])

    def as_dict(self) -> dict:
        o = self.offsets
        return {tuple(int(x) for x in self.items[o[q]:o[q + 1]]): int(self.supports[q])
                for q in range(len(self))}

    def canonical_bytes(self) -> bytes:
        return (np.ascontiguousarray(self.offsets, dtype="<u8").tobytes()
                + np.ascontiguousarray(self.items, dtype="<u4").tobytes()
                + np.ascontiguousarray(self.supports, dtype="<u8").tobytes())

    def sha256(self) -> str:
        return hashlib.sha256(self.canonical_bytes()).hexdigest()


def fim_result_sizes(ctx) -> tuple[int, int]:
    ns, ni = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.fim_fetch_results(ctx, ctypes.byref(ns), ctypes.byref(ni), None, None, None, 0, 0, 0),
           "fim_fetch_results")
    return int(ns.value), int(ni.value)


def fim_fetch_results(ctx, out=None) -> Itemsets:
    """Canonical results into new host arrays, or into `out` = (offsets, items,
    supports) buffers (numpy, pinned host or torch CUDA tensors)."""
    R, T = fim_result_sizes(ctx)
    if out is None:
        out = (np.empty(R + 1, np.uint64), np.empty(max(T, 1), np.uint32), np.empty(max(R, 1), np.uint32))
    off, it, sup = out
    _sync_torch(off, it, sup)
    po, dev = _ptr(off)
    pi, _ = _ptr(it)
    ps, _ = _ptr(sup)
    ns, ni = ctypes.c_uint64(), ctypes.c_uint64()
    cap_sets = min(int(sup.shape[0]), int(off.shape[0]) - 1)
    _check(_lib.fim_fetch_results(ctx, ctypes.byref(ns), ctypes.byref(ni), po, pi, ps, cap_sets,
                                  int(it.shape[0]), FIM_OUTPUT_DEVICE if dev else FIM_OUTPUT_HOST),
           "fim_fetch_results")
    if dev:
        return Itemsets(off[: R + 1], it[:T], sup[:R])
    return Itemsets(off[: R + 1].copy(), it[:T].copy(), sup[:R].copy())


FIM_MAX_SHARDS = 1024


def fim_mine_shard(ctx, minsup: int, flags: int, shard: int, n_shards: int) -> None:
    """fim_mine restricted to one shard's root classes (include/fim.h)."""
    _check(_lib.fim_mine_shard(ctx, int(minsup), int(flags), int(shard), int(n_shards)), "fim_mine_shard")


def fim_merge_results(ctx, n_trans: int, n_items: int, parts) -> None:
    """Replace the held itemsets with the canonical union of disjoint parts,
    each an Itemsets or an (offsets, items, supports) triple -- all numpy
    (host) or all torch CUDA tensors on the ctx's device."""
    parts = [(p.offsets, p.items, p.supports) if hasattr(p, "offsets") else tuple(p) for p in parts]
    if not parts:
        raise ValueError("fim_merge_results needs at least one part")
    flat = [a for p in parts for a in p]
    _sync_torch(*flat)
    ptrs = [_ptr(a) for a in flat]
    dev = ptrs[0][1]
    if any(d != dev for _, d in ptrs):
        raise ValueError("fim_merge_results: parts must all be host or all device")
    n = len(parts)
    n_sets = (ctypes.c_uint64 * n)(*[int(p[0].shape[0]) - 1 for p in parts])
    n_items_total = (ctypes.c_uint64 * n)(*[int(p[0][-1]) if int(p[0].shape[0]) > 1 else 0 for p in parts])
    offs = (ctypes.c_void_p * n)(*[ptrs[3 * i][0] for i in range(n)])
    its = (ctypes.c_void_p * n)(*[ptrs[3 * i + 1][0] for i in range(n)])
    sups = (ctypes.c_void_p * n)(*[ptrs[3 * i + 2][0] for i in range(n)])
    _check(_lib.fim_merge_results(ctx, int(n_trans), int(n_items), n, n_sets, n_items_total, offs, its, sups,
                                  FIM_INPUT_DEVICE if dev else FIM_INPUT_HOST), "fim_merge_results")


FIM_RULES_MAX_LEN = 20


@dataclasses.dataclass
class Rules:
    """Association rules X -> Z \\ X of the held itemsets (include/fim.h):
    set_index = index of Z in fim_fetch_results' order, ante_mask bit i = the
    i-th item of Z is in X."""
    set_index: np.ndarray  # uint64[N]
    ante_mask: np.ndarray  # uint32[N]
    conf: np.ndarray       # float64[N]
    lift: np.ndarray       # float64[N]

    def __len__(self) -> int:
        return int(self.set_index.shape[0])


def fim_rules(ctx, min_conf_ppm: int, max_len: int = 0) -> int:
    """Build the rules with confidence >= min_conf_ppm / 10^6 on the device;
    returns their number."""
    n = ctypes.c_uint64()
    _check(_lib.fim_rules(ctx, int(min_conf_ppm), int(max_len), ctypes.byref(n)), "fim_rules")
    return int(n.value)


def fim_rules_evaluated(ctx) -> int:
    """Candidate rules the last fim_rules tested (sum of 2^|Z| - 2)."""
    n = ctypes.c_uint64()
    _check(_lib.fim_rules_evaluated(ctx, ctypes.byref(n)), "fim_rules_evaluated")
    return int(n.value)


def fim_fetch_rules(ctx, out=None) -> Rules:
    """The rules of the last fim_rules into new host arrays, or into `out` =
    (set_index, ante_mask, conf, lift) buffers (numpy, pinned host or torch
    CUDA tensors)."""
    n = ctypes.c_uint64()
    _check(_lib.fim_fetch_rules(ctx, ctypes.byref(n), None, None, None, None, 0, 0), "fim_fetch_rules")
    N = int(n.value)
    if out is None:
        out = (np.empty(max(N, 1), np.uint64), np.empty(max(N, 1), np.uint32),
               np.empty(max(N, 1), np.float64), np.empty(max(N, 1), np.float64))
    si, am, cf, lf = out
    _sync_torch(si, am, cf, lf)
    ptrs = [_ptr(a) for a in out]
    dev = ptrs[0][1]
    if any(d != dev for _, d in ptrs):
        raise ValueError("fim_fetch_rules: buffers must all be host or all device")
    cap = min(int(a.shape[0]) for a in out)
    _check(_lib.fim_fetch_rules(ctx, ctypes.byref(n), *[p for p, _ in ptrs], cap,
                                FIM_OUTPUT_DEVICE if dev else FIM_OUTPUT_HOST), "fim_fetch_rules")
    if dev:
        return Rules(si[:N], am[:N], cf[:N], lf[:N])
    return Rules(si[:N].copy(), am[:N].copy(), cf[:N].copy(), lf[:N].copy())


def fim_probe(ctx, which: int) -> float:
    """Measurement probe: 0 = AND/popc word pairs per second, 1 = L2 read GB/s,
    2 / 3 = tcgen05 kind::f8f6f4 TFLOP/s with A from tensor / shared memory (N = 256),
    4 / 5 = the same with A from shared memory at N = 128 / 64."""
    r = ctypes.c_double()
    _check(_lib.fim_probe(ctx, int(which), ctypes.byref(r)), "fim_probe")
    return float(r.value)


def fim_set_tuning(ctx, key: str, value: int) -> None:
    _check(_lib.fim_set_tuning(ctx, key.encode(), int(value)), f"fim_set_tuning({key})")


def fim_pair_supports_noalloc(indptr, indices, n_items: int, out, stream=None) -> None:
    """Allocation-free singleton and pair supports (include/fim.h): device CSR
    tensors in, the caller's device uint32/int32 n_items x n_items matrix out.
    For callers that must not allocate device memory; see the header for the
    static scratch limit and the one-time per-device set-up."""
    p, dev = _ptr(indptr)
    q, dev2 = _ptr(indices)
    o, dev3 = _ptr(out)
    if not (dev and dev2 and dev3):
        raise ValueError("fim_pair_supports_noalloc takes device buffers")
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    n = int(indptr.shape[0]) - 1
    _check(_lib.fim_pair_supports_noalloc(p, q, n, int(n_items), o, s), "fim_pair_supports_noalloc")


class BatchDescriptor:
    """The fim_db_desc table of a batch, marshalled once: dbs is a sequence of
    objects with .indptr/.indices (numpy host arrays or torch CUDA tensors)
    and .m; minsups one absolute threshold per database.  Keeps the arrays
    alive; pass it to fim_mine_batched in place of (dbs, minsups) to skip the
    per-call marshalling."""

    def __init__(self, dbs, minsups):
        n = len(dbs)
        self.n = n
        self.arr = (fim_db_desc * max(1, n))()
        self.keep = []
        self.on_dev = None
        self.csr = None  # 0 (wide) or FIM_CSR_COMPACT, the same for every database
        for i, (c, ms) in enumerate(zip(dbs, minsups)):
            ip, ix = c.indptr, c.indices
            if not hasattr(ip, "data_ptr"):
                ip, ix = np.asarray(ip), np.asarray(ix)
                if (ip.dtype, ix.dtype) != (np.dtype(np.uint32), np.dtype(np.uint16)):
                    ip = np.ascontiguousarray(ip, dtype=np.int64)
                    ix = np.ascontiguousarray(ix, dtype=np.int32)
                else:
                    ip, ix = np.ascontiguousarray(ip), np.ascontiguousarray(ix)
            p, dev = _ptr(ip)
            q, _ = _ptr(ix)
            if self.on_dev is None:
                self.on_dev = dev
            elif self.on_dev != dev:
                raise ValueError("all databases must be host or all device")
            fmt = _csr_format(ip, ix)
            if self.csr is None:
                self.csr = fmt
            elif self.csr != fmt:
                raise ValueError("all databases must be wide or all compact")
            self.keep.append((ip, ix))
            self.arr[i] = fim_db_desc(p, q, int(ip.shape[0]) - 1, int(c.m), 0, int(ms))


def fim_mine_batched(ctx, dbs, minsups=None, flags: int = 0) -> None:
    """Mine many independent databases in one batched pass.  dbs: a
    BatchDescriptor, or a sequence of databases with minsups (one absolute
    threshold per database)."""
    desc = dbs if isinstance(dbs, BatchDescriptor) else BatchDescriptor(dbs, minsups)
    f = int(flags) | (FIM_INPUT_DEVICE if desc.on_dev else 0) | (desc.csr or 0)
    if desc.on_dev and desc.keep:
        _sync_torch(desc.keep[0][0])
    _check(_lib.fim_mine_batched(ctx, desc.n, ctypes.cast(desc.arr, ctypes.c_void_p), f), "fim_mine_batched")


FIM_ALL_DBS = -1


def fim_batch_sizes(ctx, db: int) -> tuple[int, int]:
    ns, ni = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.fim_fetch_batched(ctx, int(db), ctypes.byref(ns), ctypes.byref(ni), None, None, None, 0, 0, 0),
           "fim_fetch_batched")
    return int(ns.value), int(ni.value)


def fim_fetch_batched(ctx, db: int, out=None) -> Itemsets:
    """Canonical results of database `db` of the last batch (FIM_ALL_DBS: every
    database, in database order), into new host arrays or `out` buffers
    (numpy, pinned host or torch CUDA tensors)."""
    R, T = fim_batch_sizes(ctx, db)
    if out is None:
        out = (np.empty(R + 1, np.uint64), np.empty(max(T, 1), np.uint32), np.empty(max(R, 1), np.uint32))
    off, it, sup = out
    _sync_torch(off, it, sup)
    po, dev = _ptr(off)
    pi, _ = _ptr(it)
    ps, _ = _ptr(sup)
    ns, ni = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.fim_fetch_batched(ctx, int(db), ctypes.byref(ns), ctypes.byref(ni), po, pi, ps,
                                  min(int(sup.shape[0]), int(off.shape[0]) - 1), int(it.shape[0]),
                                  FIM_OUTPUT_DEVICE if dev else FIM_OUTPUT_HOST), "fim_fetch_batched")
    if dev:
        return Itemsets(off[: R + 1], it[:T], sup[:R])
    return Itemsets(off[: R + 1], it[:T], sup[:R])


def fim_batch_slices(ctx, n_db: int) -> np.ndarray:
    s = np.empty(n_db + 1, np.uint64)
    _check(_lib.fim_batch_slices(ctx, s.ctypes.data, n_db + 1), "fim_batch_slices")
    return s


def fim_sched_load_weights(ctx, weights) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(_lib.fim_sched_load_weights(ctx, w.ctypes.data, w.size), "fim_sched_load_weights")


def fim_fetch_traces(ctx):
    """(features float32 [n, 8], targets float32 [n, 2]) of the last FIM_TRACE mine."""
    n = ctypes.c_uint64()
    _check(_lib.fim_fetch_traces(ctx, ctypes.byref(n), None, None, 0), "fim_fetch_traces")
    x = np.zeros((n.value, 8), np.float32)
    t = np.zeros((n.value, 2), np.float32)
    if n.value:
        _check(_lib.fim_fetch_traces(ctx, ctypes.byref(n), x.ctypes.data, t.ctypes.data, n.value),
               "fim_fetch_traces")
    return x, t


def fim_mlp_forward(ctx, params, x, y, cache=None, bf16=False) -> None:
    """Device tensors: params [4866], x [B, 8] -> y [B, 2]; cache [B, 256] or None."""
    _sync_torch(params)
    _check(_lib.fim_mlp_forward(ctx, params.data_ptr(), x.data_ptr(), int(x.shape[0]), y.data_ptr(),
                                cache.data_ptr() if cache is not None else None, int(bool(bf16))),
           "fim_mlp_forward")


def fim_mlp_backward(ctx, params, x, y, t, cache, grad, bf16=False) -> float:
    """Device tensors; writes grad [4866]; returns the mean loss."""
    loss = ctypes.c_float()
    _sync_torch(params)
    _check(_lib.fim_mlp_backward(ctx, params.data_ptr(), x.data_ptr(), y.data_ptr(), t.data_ptr(),
                                 cache.data_ptr(), int(x.shape[0]), grad.data_ptr(), ctypes.byref(loss),
                                 int(bool(bf16))), "fim_mlp_backward")
    return float(loss.value)


def fim_mlp_adam(ctx, params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    _sync_torch(params)
    _check(_lib.fim_mlp_adam(ctx, params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), int(step),
                             float(lr), float(beta1), float(beta2), float(eps)), "fim_mlp_adam")


def fim_get_stats(ctx) -> dict:
    s = fim_stats()
    _check(_lib.fim_get_stats(ctx, ctypes.byref(s)), "fim_get_stats")
    return s.as_dict()


def mine(indptr, indices, n_items: int, minsup: int, flags: int = 0, device: int = 0) -> Itemsets:
    """One-shot convenience: build, mine and fetch in a fresh context."""
    ctx = fim_create(device)
    try:
        fim_build_bitmaps(ctx, indptr, indices, n_items)
        fim_mine(ctx, minsup, flags)
        return fim_fetch_results(ctx)
    finally:
        fim_destroy(ctx)
