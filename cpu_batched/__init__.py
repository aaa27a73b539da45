"""CPU comparator: the paper's own CPU design of the seeding stage, for timing next to the GPU.

Algorithm 3 over batches of reads with one FIFO queue and prefetching of the occurrence blocks
each queued entry will read, 64-byte blocks of 128 rows, a 10-mer ds-interval table, and
BatchLocate with prefetching (Sections 2.2-2.5, Algorithms 2 and 3), OpenMP over batches.  It
is context for the GPU numbers, not the oracle (the tests check it against the oracle) and not
part of the library: nothing in the GPU path calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libcpu_batched.so")
_lock = threading.Lock()
_lib = None

SMEM_DTYPE = np.dtype([("read", np.uint64), ("qbeg", np.uint64), ("qend", np.uint64),
                       ("k", np.uint64), ("kr", np.uint64), ("s", np.uint64)])


def build(force: bool = False) -> str:
    """Compile cpu_batched.cpp into _build/libcpu_batched.so (g++ -O3, OpenMP)."""
    src = os.path.join(_HERE, "cpu_batched.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O3", "-std=c++17", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            sig = {
                "cb_index_build": ([P, U64, U64, P, U32, I], P),
                "cb_index_free": ([P], None),
                "cb_seed": ([P, P, P, U32, U32, U32, U32, U32, I], P),
                "cb_result_nsmem": ([P], U64),
                "cb_result_nhits": ([P], U64),
                "cb_result_get": ([P, P, P], None),
                "cb_result_free": ([P], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


class Index:
    """From the BWT (n bytes: 0 = $, 1..4 = A..T), the row of $ and the sampled suffix array."""

    def __init__(self, bwt: np.ndarray, primary: int, ssa: np.ndarray, sa_rate: int = 32, threads: int = 0):
        bwt = np.ascontiguousarray(bwt, dtype=np.uint8)
        ssa = np.ascontiguousarray(ssa, dtype=np.uint32)
        self.n = len(bwt)
        self._h = lib().cb_index_build(_p(bwt), self.n, primary, _p(ssa), sa_rate, threads)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().cb_index_free(self._h)
            self._h = None

    def seed(self, seq, off, min_len: int = 19, min_occ: int = 1, max_occ: int = 500, batch: int = 4096,
             threads: int = 0):
        """(records, hits): records of SMEM_DTYPE per read in qbeg order, hits of the records with
        s <= max_occ in record order, then SA-row order."""
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        h = lib().cb_seed(self._h, _p(seq), _p(off), len(off) - 1, min_len, min_occ, max_occ, batch, threads)
        try:
            ns, nh = lib().cb_result_nsmem(h), lib().cb_result_nhits(h)
            sm = np.empty(max(ns, 1) * 6, np.uint64)
            hits = np.empty(max(nh, 1), np.uint32)
            lib().cb_result_get(h, _p(sm), _p(hits))
        finally:
            lib().cb_result_free(h)
        return sm[:ns * 6].view(SMEM_DTYPE).reshape(-1), hits[:nh]
