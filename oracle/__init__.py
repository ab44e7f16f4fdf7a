"""CPU oracle for the Boolean-matrix frequent-itemset miner -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (the CUDA library and its Python
binding) never imports, links or calls it, and this package imports nothing
from the product path.

Contents
  apriori(...)        plain level-wise Apriori in C (oracle/apriori.c),
                      counting by direct transaction scans (Eq. 1-3)
  support_many(...)   S(X) of given itemsets by a direct scan (Eq. 2)
  mlp                 float64 reference of the 8-64-64-2 scheduling MLP
Parity status: apriori and support_many are pinned by brute force, closed
forms and library cross-checks in tests/test_oracle.py; the MLP reference is
pinned by finite differences and closed forms in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile oracle/apriori.c with gcc into oracle/_build/liboracle.so.

    ``mutant`` > 0 builds a copy with one planted mistake (see OR_MUTANT in
    apriori.c); only the tests that check the pins' sensitivity ask for it.
    """
    src = os.path.join(_HERE, "apriori.c")
    so = _SO if not mutant else _SO.replace(".so", f"_mut{int(mutant)}.so")
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(src)):
        return so
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-pthread", f"-DOR_MUTANT={int(mutant)}", src, "-o", tmp])
    os.replace(tmp, so)
    return so


class _Result(ctypes.Structure):
    _fields_ = [("n_sets", ctypes.c_uint64), ("n_items_total", ctypes.c_uint64),
                ("offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("items", ctypes.POINTER(ctypes.c_uint32)),
                ("supports", ctypes.POINTER(ctypes.c_uint64)),
                ("n_candidates", ctypes.c_uint64), ("max_level", ctypes.c_int)]


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.or_apriori.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(_Result)]
    lib.or_apriori.restype = ctypes.c_int
    lib.or_free.argtypes = [ctypes.POINTER(_Result)]
    lib.or_free.restype = None
    lib.or_support_many.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, P, P,
                                    ctypes.c_uint64, ctypes.c_int, P]
    lib.or_support_many.restype = ctypes.c_int
    return lib


def _load(mutant: int = 0):
    global _lib
    if mutant:
        return _bind(build(mutant=mutant))
    if _lib is None:
        _lib = _bind(build())
    return _lib


@dataclasses.dataclass
class Itemsets:
    """Canonical list of frequent itemsets: set q is items[offsets[q]:offsets[q+1]]."""
    offsets: np.ndarray   # uint64[R+1]
    items: np.ndarray     # uint32[sum |X|]
    supports: np.ndarray  # uint64[R]
    n_candidates: int = 0
    max_level: int = 0

    def __len__(self) -> int:
        return int(self.supports.shape[0])

    def as_dict(self) -> dict:
        o = self.offsets
        return {tuple(int(x) for x in self.items[o[q]:o[q + 1]]): int(self.supports[q])
                for q in range(len(self))}

    def canonical_bytes(self) -> bytes:
        """Byte stream used for bit-exact comparison: offsets, items, supports."""
        return (np.ascontiguousarray(self.offsets, dtype="<u8").tobytes()
                + np.ascontiguousarray(self.items, dtype="<u4").tobytes()
                + np.ascontiguousarray(self.supports, dtype="<u8").tobytes())

    def sha256(self) -> str:
        return hashlib.sha256(self.canonical_bytes()).hexdigest()


def _threads(n: int | None) -> int:
    if n:
        return int(n)
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def apriori(indptr, indices, m: int, threshold: int, strict: bool = False,
            threads: int | None = None, max_len: int = 0, _mutant: int = 0) -> Itemsets:
    """All frequent itemsets of the CSR database (plain Apriori, Eq. 1-3).

    ``threshold`` is an absolute count; frequent means S >= threshold, or the
    paper's literal S > threshold with ``strict``.  Raises ValueError on a
    malformed CSR (non-monotone indptr, item outside [0, m)).
    """
    lib = _load(_mutant)
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    res = _Result()
    rc = lib.or_apriori(ip.ctypes.data, ix.ctypes.data, ip.shape[0] - 1, int(m),
                        int(threshold), int(bool(strict)), _threads(threads), int(max_len),
                        ctypes.byref(res))
    if rc == -1:
        raise ValueError("malformed transaction database")
    if rc != 0:
        raise MemoryError(f"oracle failed with code {rc}")
    try:
        R, T = res.n_sets, res.n_items_total
        off = np.ctypeslib.as_array(res.offsets, shape=(R + 1,)).copy()
        items = (np.ctypeslib.as_array(res.items, shape=(T,)).copy() if T
                 else np.zeros(0, np.uint32))
        sup = (np.ctypeslib.as_array(res.supports, shape=(R,)).copy() if R
               else np.zeros(0, np.uint64))
        return Itemsets(off, items, sup, int(res.n_candidates), int(res.max_level))
    finally:
        lib.or_free(ctypes.byref(res))


def support_many(indptr, indices, m: int, itemsets, threads: int | None = None) -> np.ndarray:
    """S(X) for every itemset in ``itemsets`` (a list of item sequences)."""
    lib = _load()
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    lens = [len(x) for x in itemsets]
    qoff = np.zeros(len(itemsets) + 1, dtype=np.uint64)
    np.cumsum(lens, out=qoff[1:])
    qitems = np.asarray([int(v) for x in itemsets for v in x], dtype=np.uint32)
    if qitems.size == 0:
        qitems = np.zeros(1, np.uint32)
    out = np.zeros(max(1, len(itemsets)), dtype=np.uint64)
    rc = lib.or_support_many(ip.ctypes.data, ix.ctypes.data, ip.shape[0] - 1, int(m),
                             qoff.ctypes.data, qitems.ctypes.data, len(itemsets),
                             _threads(threads), out.ctypes.data)
    if rc == -1:
        raise ValueError("malformed transaction database or query")
    if rc != 0:
        raise MemoryError(f"oracle failed with code {rc}")
    return out[: len(itemsets)]
