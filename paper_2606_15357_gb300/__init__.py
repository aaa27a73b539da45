"""Seeding stage of minibwa (arxiv 2606.15357) on one GB300 GPU: Python binding.

This module only marshals arguments for ``libminibwa_gpu.so`` (C ABI declared in
``include/minibwa_gpu.h``); every step of the computation runs in its CUDA
kernels.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
pointers are passed through unchanged and the library stages host buffers.
There is no CPU fallback: if the library has not been built, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .nvcc_build import SO, build

__all__ = ["SMEM_DTYPE", "Opts", "MbError", "lib", "build", "Index", "mb_index_build",
           "mb_index_load", "mb_seed_batch", "mb_locate", "mb_bs_filter", "seed"]

MB_BS3, MB_BATCHED, MB_CHECKED, MB_NO_KMER, MB_COUNT = 0x1, 0x2, 0x4, 0x8, 0x10
MB_NO_AUX, MB_STEP_ONLY, MB_SMEM_ONE_LOOP, MB_LOCATE_JOIN, MB_LOCATE_AUX = 0x20, 0x40, 0x80, 0x100, 0x200
AUX_RATE = 4   # sample rate of the auxiliary SA / ISA samples (mb_index_export_aux)
MB_SMEM_OVER_MAX_OCC, MB_SMEM_ROUND2 = 0x1, 0x2
MB_ERR_CAPACITY = -3

SMEM_DTYPE = np.dtype([("read", "<u4"), ("qbeg", "<u4"), ("qend", "<u4"), ("flags", "<u4"),
                       ("k", "<u8"), ("kr", "<u8"), ("s", "<u8"), ("hit_off", "<u8")])
assert SMEM_DTYPE.itemsize == 48


class Opts(ctypes.Structure):
    """mb_opts; zero fields take the library defaults (l=19, c=1, max_occ=500, r=32, k=10)."""
    _fields_ = [("min_len", ctypes.c_uint32), ("min_occ", ctypes.c_uint32),
                ("max_occ", ctypes.c_uint32), ("sa_rate", ctypes.c_uint32),
                ("kmer_k", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("chunk_reads", ctypes.c_uint32), ("prefetch_depth", ctypes.c_uint32),
                ("block_size", ctypes.c_uint32), ("smem_burst", ctypes.c_uint32),
                ("smem_wait", ctypes.c_uint32), ("smem_warps", ctypes.c_uint32),
                ("smem_reads_per_warp", ctypes.c_uint32)]


class MbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load libminibwa_gpu.so.  Raises if it was not built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                raise RuntimeError(f"libminibwa_gpu.so is not built ({SO}); "
                                   "run `python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(SO)
            P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            PP = ctypes.POINTER(ctypes.c_void_p)
            PU64 = ctypes.POINTER(ctypes.c_uint64)
            OP = ctypes.POINTER(Opts)
            sig = {
                "mb_index_build": ([P, U64, OP, U64, P, PP], I),
                "mb_index_save": ([P, ctypes.c_char_p], I),
                "mb_index_load": ([ctypes.c_char_p, P, PP], I),
                "mb_index_free": ([P], None),
                "mb_index_info": ([P, PU64, PU64, PU64], I),
                "mb_index_export": ([P, P, P, P, P, P, P], I),
                "mb_index_drop_sa": ([P], I),
                "mb_index_export_aux": ([P, P, P, P], I),
                "mb_index_kmer_get": ([P, P, U64, P], I),
                "mb_seed_batch": ([P, P, P, U32, P, OP, P, P, U64, PU64, PU64], I),
                "mb_locate": ([P, P, U64, OP, P, P, U64, PU64], I),
                "mb_seed_locate": ([P, P, P, U32, P, OP, P, P, U64, P, U64, PU64, PU64], I),
                "mb_bs_filter": ([P, P, U64, P, P, U64, P, P], I),
                "mb_hit_to_ref": ([P, U64, U64, ctypes.POINTER(I), PU64], I),
                "mb_bs_split": ([P, P, P, P, U32, P, P, U64, P, P, U64, OP, P, P, U64, PU64], I),
                "mb_rescue_prefilter": ([P, P, P, P, U32, U32, P, P], I),
                "mb_strerror": ([I], ctypes.c_char_p),
                "mb_last_error": ([], ctypes.c_char_p),
                "mb_device_extent": ([P, PU64, PU64], I),
                "mb_index_l2_persist": ([P, P, U64, PU64], I),
                "mb_seed_batch_noalloc": ([P, P, P, U32, P, OP, P, P, U64, PU64, PU64], I),
                "mb_reseed": ([P, P, P, U32, P, P, U64, OP, P, P, U64, PU64, PU64], I),
                "mb_plan_create": ([P, OP, U32, U64, U64, U64, PP], I),
                "mb_plan_run": ([P, P, P, U32, P, P], I),
                "mb_plan_result": ([P, P, PP, PU64, PP, PU64], I),
                "mb_plan_free": ([P], None),
                "mb_plan_copy": ([P, P, P, U64, P, U64], I),
                "mb_plan_capture": ([P, P, P, U32, P], I),
                "mb_plan_replay": ([P, P], I),
                "mb_autotune": ([P, P, P, U32, OP, P, OP, ctypes.POINTER(ctypes.c_double)], I),
                "mb_autotune_points": ([P, P, P, U32, OP, P, OP, ctypes.POINTER(ctypes.c_double), OP,
                                        ctypes.POINTER(ctypes.c_double), U32, ctypes.POINTER(U32)], I),
                "mb_serve_create": ([P, OP, U64, PP], I),
                "mb_serve_submit": ([P, P, P, U32, PU64], I),
                "mb_serve_poll": ([P, U64, ctypes.POINTER(I)], I),
                "mb_serve_wait": ([P, U64, U32, PP, PU64, PP, PU64, ctypes.POINTER(ctypes.c_double)], I),
                "mb_serve_release": ([P, U64], I),
                "mb_serve_destroy": ([P], I),
                "mb_serve_stats": ([P, ctypes.POINTER(U32), PU64, PU64], I),
                "mb_serve_counters": ([P, P, U32], I),
                "mb_serve_inject": ([P, ctypes.c_int64, U32], I),
                "mb_set_l2_fetch_granularity": ([I, ctypes.POINTER(I)], I),
                "mb_profile_enable": ([I], None),
                "mb_profile_get": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), PU64], I),
                "mb_profile_reset": ([], None),
                "mb_launch_count": ([], U64),
                "mb_work_counters": ([PU64, PU64, PU64, PU64, PU64], None),
                "mb_work_counters_all": ([P, U32], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        raise MbError(rc, f"{what}: {L.mb_strerror(rc).decode()}: {L.mb_last_error().decode()}")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(type(x))


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _opts(opts) -> Opts:
    if opts is None:
        return Opts()
    if isinstance(opts, Opts):
        return opts
    return Opts(**opts)


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


class Index:
    """A device-resident FMD-index (handle to mb_index)."""

    def __init__(self, handle):
        self._h = handle
        n, prim, rl = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().mb_index_info(handle, ctypes.byref(n), ctypes.byref(prim), ctypes.byref(rl)),
               "mb_index_info")
        self.n, self.primary, self.ref_len = n.value, prim.value, rl.value

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            lib().mb_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def save(self, path: str):
        _check(lib().mb_index_save(self._h, path.encode()), "mb_index_save")

    def drop_sa(self):
        _check(lib().mb_index_drop_sa(self._h), "mb_index_drop_sa")

    def export(self, sa=False, bwt=False, ssa=False, occ=False, kmer=False, sa_rate=32, kmer_k=10):
        """Copy index arrays to host numpy arrays (for tests)."""
        n = self.n
        out = {}
        a_sa = np.empty(n, np.uint32) if sa else None
        a_bwt = np.empty(n, np.uint8) if bwt else None
        a_ssa = np.empty((n + sa_rate - 1) // sa_rate, np.uint32) if ssa else None
        a_occ = np.empty((n // 64 + 1) * 4, np.uint64) if occ else None
        a_kmer = np.empty(3 * 4 ** kmer_k, np.uint32) if kmer else None
        C = np.empty(5, np.uint64)
        _check(lib().mb_index_export(self._h, _ptr(a_sa), _ptr(a_bwt), _ptr(a_ssa), _ptr(a_occ),
                                     _ptr(a_kmer), _ptr(C)), "mb_index_export")
        for k, v in (("sa", a_sa), ("bwt", a_bwt), ("ssa", a_ssa), ("occ", a_occ), ("kmer", a_kmer)):
            if v is not None:
                out[k] = v
        out["C"] = C
        return out

    def export_aux(self):
        """(text2, sa_aux, isa_aux) as host arrays (see mb_index_export_aux)."""
        n = self.n
        t2 = np.empty((n - 1 + 15) // 16 + 2, np.uint32)
        sx = np.empty((n + AUX_RATE - 1) // AUX_RATE, np.uint32)
        ix = np.empty((n + AUX_RATE - 1) // AUX_RATE, np.uint32)
        _check(lib().mb_index_export_aux(self._h, _ptr(t2), _ptr(sx), _ptr(ix)), "mb_index_export_aux")
        return t2, sx, ix

    def kmer_get(self, codes) -> np.ndarray:
        """(k, kr, s) of the k-mer table for each k-mer code, as an (n, 3) array (mb_index_kmer_get)."""
        codes = np.ascontiguousarray(codes, dtype=np.uint64)
        out = np.empty((len(codes), 3), np.uint32)
        _check(lib().mb_index_kmer_get(self._h, _ptr(codes), len(codes), _ptr(out)), "mb_index_kmer_get")
        return out

    def l2_persist(self, max_bytes: int, stream=None) -> int:
        """Access-policy window over the k-mer table on `stream` (mb_index_l2_persist); returns the
        window's bytes (0 removes it)."""
        w = ctypes.c_uint64()
        _check(lib().mb_index_l2_persist(self._h, _stream(stream), max_bytes, ctypes.byref(w)),
               "mb_index_l2_persist")
        return w.value

    def hit_to_ref(self, pos: int, length: int):
        strand, rpos = ctypes.c_int(), ctypes.c_uint64()
        _check(lib().mb_hit_to_ref(self._h, pos, length, ctypes.byref(strand), ctypes.byref(rpos)),
               "mb_hit_to_ref")
        return strand.value, rpos.value


def mb_index_build(ref, opts=None, n_seed: int = 0, stream=None) -> Index:
    """FMD-index of `ref` (uint8 codes, host numpy or torch tensor) built on the GPU."""
    o = _opts(opts)
    h = ctypes.c_void_p()
    _check(lib().mb_index_build(_ptr(ref), int(ref.numel() if hasattr(ref, "numel") else len(ref)),
                                ctypes.byref(o), n_seed, _stream(stream), ctypes.byref(h)),
           "mb_index_build")
    return Index(h)


def mb_index_load(path: str, stream=None) -> Index:
    h = ctypes.c_void_p()
    _check(lib().mb_index_load(path.encode(), _stream(stream), ctypes.byref(h)), "mb_index_load")
    return Index(h)


def mb_seed_batch(index: Index, seq, off, mate=None, opts=None, stream=None, out=None, cap=None):
    """SMEMs of a batch of reads.  Returns (records, n_smem, n_hits).

    With `out` None the records come back as a host numpy array of SMEM_DTYPE;
    otherwise they are written into `out` (a uint8 buffer of cap*48 bytes,
    host or device) and `out` is returned.
    """
    o = _opts(opts)
    n_reads = (off.numel() if hasattr(off, "numel") else len(off)) - 1
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    if out is None:
        cap = cap if cap is not None else max(16, 8 * n_reads)
        while True:
            buf = np.empty(cap, dtype=SMEM_DTYPE)
            rc = lib().mb_seed_batch(index.handle, _ptr(seq), _ptr(off), n_reads, _ptr(mate),
                                     ctypes.byref(o), _stream(stream), _ptr(buf), cap,
                                     ctypes.byref(n_out), ctypes.byref(n_hits))
            if rc == MB_ERR_CAPACITY:
                cap = n_out.value
                continue
            _check(rc, "mb_seed_batch")
            return buf[:n_out.value], n_out.value, n_hits.value
    rc = lib().mb_seed_batch(index.handle, _ptr(seq), _ptr(off), n_reads, _ptr(mate), ctypes.byref(o),
                             _stream(stream), _ptr(out), cap, ctypes.byref(n_out), ctypes.byref(n_hits))
    _check(rc, "mb_seed_batch")
    return out, n_out.value, n_hits.value


def mb_locate(index: Index, smem, n_smem: int, opts=None, stream=None, hits=None, cap=None):
    """Text positions of the hits of every SMEM not over max_occ.  Returns (hits, n_hits)."""
    o = _opts(opts)
    n_hits = ctypes.c_uint64()
    if hits is None:
        cap = 0 if cap is None else cap
        while True:
            buf = np.empty(max(cap, 1), dtype=np.uint32)
            rc = lib().mb_locate(index.handle, _ptr(smem), n_smem, ctypes.byref(o), _stream(stream),
                                 _ptr(buf), cap, ctypes.byref(n_hits))
            if rc == MB_ERR_CAPACITY:
                cap = n_hits.value
                continue
            _check(rc, "mb_locate")
            return buf[:n_hits.value], n_hits.value
    _check(lib().mb_locate(index.handle, _ptr(smem), n_smem, ctypes.byref(o), _stream(stream),
                           _ptr(hits), cap, ctypes.byref(n_hits)), "mb_locate")
    return hits, n_hits.value


def mb_bs_filter(index: Index, smem, n_smem: int, mate, hits, n_hits: int, stream=None, keep=None):
    """Section 2.9 strand rule: 1 for hits kept, 0 for hits dropped."""
    if keep is None:
        keep = np.empty(max(n_hits, 1), dtype=np.uint8)
    _check(lib().mb_bs_filter(index.handle, _ptr(smem), n_smem, _ptr(mate), _ptr(hits), n_hits,
                              _stream(stream), _ptr(keep)), "mb_bs_filter")
    return keep[:n_hits]


PIECE_DTYPE = np.dtype([("hit", np.uint64), ("read", np.uint32), ("qbeg", np.uint32),
                        ("qend", np.uint32), ("pos", np.uint32)])


def mb_bs_split(index: Index, ref, seq, off, mate, smem, n_smem: int, hits, n_hits: int, keep=None,
                opts=None, stream=None):
    """Section 2.9 T-to-C split of bisulfite seed hits; returns a host array of PIECE_DTYPE."""
    o = _opts(opts)
    n_reads = (off.numel() if hasattr(off, "numel") else len(off)) - 1
    n = ctypes.c_uint64()
    cap = 0
    while True:
        buf = np.empty(max(cap, 1), dtype=PIECE_DTYPE)
        rc = lib().mb_bs_split(index.handle, _ptr(ref), _ptr(seq), _ptr(off), n_reads, _ptr(mate), _ptr(smem),
                               n_smem, _ptr(hits), _ptr(keep), n_hits, ctypes.byref(o), _stream(stream),
                               _ptr(buf), cap, ctypes.byref(n))
        if rc == MB_ERR_CAPACITY:
            cap = n.value
            continue
        _check(rc, "mb_bs_split")
        return buf[:n.value]


def mb_rescue_prefilter(reads, read_off, wins, win_off, q: int = 7, stream=None, best=None):
    """Section 2.7 mate-rescue prefilter: max_t M_t of q-mer matches per (read, window) pair."""
    n = (read_off.numel() if hasattr(read_off, "numel") else len(read_off)) - 1
    if best is None:
        best = np.empty(max(n, 1), dtype=np.uint32)
    _check(lib().mb_rescue_prefilter(_ptr(reads), _ptr(read_off), _ptr(wins), _ptr(win_off), n, q,
                                     _stream(stream), _ptr(best)), "mb_rescue_prefilter")
    return best[:n]


def mb_reseed(index: Index, seq, off, smem, n_smem: int, mate=None, opts=None, stream=None):
    """Second seeding round (Section 2.6) on first-round records; returns (records, n, n_hits)."""
    o = _opts(opts)
    n_reads = (off.numel() if hasattr(off, "numel") else len(off)) - 1
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    cap = max(16, 4 * n_smem)
    while True:
        buf = np.empty(cap, dtype=SMEM_DTYPE)
        rc = lib().mb_reseed(index.handle, _ptr(seq), _ptr(off), n_reads, _ptr(mate), _ptr(smem), n_smem,
                             ctypes.byref(o), _stream(stream), _ptr(buf), cap, ctypes.byref(n_out),
                             ctypes.byref(n_hits))
        if rc == MB_ERR_CAPACITY:
            cap = n_out.value
            continue
        _check(rc, "mb_reseed")
        return buf[:n_out.value], n_out.value, n_hits.value


def seed_locate(index: Index, seq, off, mate=None, opts=None, stream=None, out=None, cap=None, hits=None,
                hits_cap=None):
    """SMEMs and their hits in one pipelined call (host or device buffers).

    With `out` None returns host numpy arrays (records, hits), sized by a retry on
    MB_ERR_CAPACITY; otherwise writes into `out` (uint8, cap*48 bytes) and `hits` (hits_cap
    u32) and returns (n_smem, n_hits)."""
    o = _opts(opts)
    n_reads = (off.numel() if hasattr(off, "numel") else len(off)) - 1
    n_out, n_hits = ctypes.c_uint64(), ctypes.c_uint64()
    if out is None:
        cap = cap if cap is not None else max(16, 4 * n_reads)
        hits_cap = hits_cap if hits_cap is not None else max(16, 32 * n_reads)
        while True:
            buf = np.empty(max(cap, 1), dtype=SMEM_DTYPE)
            hbuf = np.empty(max(hits_cap, 1), dtype=np.uint32)
            rc = lib().mb_seed_locate(index.handle, _ptr(seq), _ptr(off), n_reads, _ptr(mate), ctypes.byref(o),
                                      _stream(stream), _ptr(buf), cap, _ptr(hbuf), hits_cap,
                                      ctypes.byref(n_out), ctypes.byref(n_hits))
            if rc == MB_ERR_CAPACITY:
                cap, hits_cap = n_out.value, n_hits.value
                continue
            _check(rc, "mb_seed_locate")
            return buf[:n_out.value], hbuf[:n_hits.value]
    _check(lib().mb_seed_locate(index.handle, _ptr(seq), _ptr(off), n_reads, _ptr(mate), ctypes.byref(o),
                                _stream(stream), _ptr(out), cap, _ptr(hits), hits_cap, ctypes.byref(n_out),
                                ctypes.byref(n_hits)), "mb_seed_locate")
    return n_out.value, n_hits.value


def seed(index: Index, seq, off, mate=None, opts=None, stream=None):
    """SMEMs then hits, host in / host out (numpy).  Returns (records, hits)."""
    sm, m, nh = mb_seed_batch(index, seq, off, mate, opts, stream)
    hits, _ = mb_locate(index, sm, m, opts, stream, cap=nh)
    return sm, hits


# ---------------------------------------------------------------------------- measurement hooks
def profile_enable(on: bool = True):
    lib().mb_profile_enable(int(on))


def profile_reset():
    lib().mb_profile_reset()


def profile_get(kernel: str):
    """(summed device ms, launches) of a timed kernel ("smem", "locate")."""
    ms, n = ctypes.c_double(), ctypes.c_uint64()
    _check(lib().mb_profile_get(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)), "mb_profile_get")
    return ms.value, n.value


def launch_count() -> int:
    return int(lib().mb_launch_count())


def work_counters() -> dict:
    v = np.zeros(10, dtype=np.uint64)
    lib().mb_work_counters_all(_ptr(v), 10)
    return dict(zip(("ext_steps", "ext_blocks", "kmer_lookups", "lf_steps", "sa_reads", "u_walk_steps",
                     "u_samples", "u_text_loads", "joins", "joins_off"), (int(x) for x in v)))


# ---------------------------------------------------------------------------- batched form
class Plan:
    """A reusable seeding plan (mb_plan_*): fixed device workspace, no host synchronization
    inside a run, capturable into a CUDA graph."""

    def __init__(self, index: Index, max_reads: int, max_bases: int, max_smem: int, max_hits: int,
                 opts=None):
        self.index = index
        self.opts = _opts(opts)
        h = ctypes.c_void_p()
        _check(lib().mb_plan_create(index.handle, ctypes.byref(self.opts), max_reads, max_bases,
                                    max_smem, max_hits, ctypes.byref(h)), "mb_plan_create")
        self._h = h

    def run(self, seq, off, mate=None, stream=None):
        n = (off.numel() if hasattr(off, "numel") else len(off)) - 1
        _check(lib().mb_plan_run(self._h, _ptr(seq), _ptr(off), n, _ptr(mate), _stream(stream)),
               "mb_plan_run")

    def capture(self, seq, off, mate=None):
        n = (off.numel() if hasattr(off, "numel") else len(off)) - 1
        _check(lib().mb_plan_capture(self._h, _ptr(seq), _ptr(off), n, _ptr(mate)), "mb_plan_capture")

    def replay(self, stream=None):
        _check(lib().mb_plan_replay(self._h, _stream(stream)), "mb_plan_replay")

    def result_ptrs(self, stream=None):
        """(smem device ptr, n_smem, hits device ptr, n_hits); raises on capacity overflow."""
        sp, hp = ctypes.c_void_p(), ctypes.c_void_p()
        ns, nh = ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib().mb_plan_result(self._h, _stream(stream), ctypes.byref(sp), ctypes.byref(ns),
                                  ctypes.byref(hp), ctypes.byref(nh))
        _check(rc, "mb_plan_result")
        return sp.value, ns.value, hp.value, nh.value

    def result(self, stream=None):
        """Records and hits of the last run as host numpy arrays."""
        sp, ns, hp, nh = self.result_ptrs(stream)
        sm = np.empty(max(ns, 1), dtype=SMEM_DTYPE)
        hits = np.empty(max(nh, 1), dtype=np.uint32)
        _check(lib().mb_plan_copy(self._h, _stream(stream), _ptr(sm), ns, _ptr(hits), nh), "mb_plan_copy")
        return sm[:ns], hits[:nh]

    def free(self):
        if getattr(self, "_h", None):
            lib().mb_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune(index: Index, seq, off, opts=None, stream=None, points: bool = False):
    """Fastest launch shape on this batch: (Opts, ms), and with points=True also the list of every
    shape tried as (Opts, ms)."""
    o = _opts(opts)
    best = Opts()
    ms = ctypes.c_double()
    n = (off.numel() if hasattr(off, "numel") else len(off)) - 1
    if not points:
        _check(lib().mb_autotune(index.handle, _ptr(seq), _ptr(off), n, ctypes.byref(o), _stream(stream),
                                 ctypes.byref(best), ctypes.byref(ms)), "mb_autotune")
        return best, ms.value
    cap = 256
    pts = (Opts * cap)()
    pms = (ctypes.c_double * cap)()
    npts = ctypes.c_uint32()
    _check(lib().mb_autotune_points(index.handle, _ptr(seq), _ptr(off), n, ctypes.byref(o), _stream(stream),
                                    ctypes.byref(best), ctypes.byref(ms), pts, pms, cap, ctypes.byref(npts)),
           "mb_autotune_points")
    return best, ms.value, [(pts[i], pms[i]) for i in range(min(npts.value, cap))]


def shape_of(o: Opts) -> dict:
    """The launch-shape fields of an Opts as a plain dict (for reports)."""
    split = not (o.flags & MB_SMEM_ONE_LOOP)
    return {"block_size": o.block_size or 256, "work_queue": bool(o.flags & MB_BATCHED),
            "smem_form": "split" if split else "one_loop",
            "smem_burst": (o.smem_burst or 8) if split else None,
            "smem_wait": (o.smem_wait or 8) if split else None,
            "smem_warps": (o.smem_warps or None) if split else None,
            "smem_reads_per_warp": (o.smem_reads_per_warp or 32) if split else None,
            "locate_walks_per_lane": o.prefetch_depth or 1, "locate_join": bool(o.flags & MB_LOCATE_JOIN),
            "locate_aux": bool(o.flags & MB_LOCATE_AUX)}


# ---------------------------------------------------------------------------- served form
class Server:
    """Continuous-batching seeding server (mb_serve_*): submit host read batches, get tickets."""

    def __init__(self, index: Index, hbm_budget: int = 4 << 30, opts=None):
        self.index = index
        self.opts = _opts(opts)
        h = ctypes.c_void_p()
        _check(lib().mb_serve_create(index.handle, ctypes.byref(self.opts), hbm_budget, ctypes.byref(h)),
               "mb_serve_create")
        self._h = h

    def submit(self, seq: np.ndarray, off: np.ndarray) -> int:
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        t = ctypes.c_uint64()
        _check(lib().mb_serve_submit(self._h, _ptr(seq), _ptr(off), len(off) - 1, ctypes.byref(t)),
               "mb_serve_submit")
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(lib().mb_serve_poll(self._h, ticket, ctypes.byref(d)), "mb_serve_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = 0, release: bool = True):
        """(records, hits, latency_ms) as host numpy arrays (copied)."""
        sp, hp = ctypes.c_void_p(), ctypes.c_void_p()
        ns, nh, lat = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
        _check(lib().mb_serve_wait(self._h, ticket, timeout_ms, ctypes.byref(sp), ctypes.byref(ns),
                                   ctypes.byref(hp), ctypes.byref(nh), ctypes.byref(lat)), "mb_serve_wait")
        sm = np.empty(ns.value, dtype=SMEM_DTYPE)
        hits = np.empty(nh.value, dtype=np.uint32)
        if ns.value:
            ctypes.memmove(sm.ctypes.data, sp.value, ns.value * 48)
        if nh.value:
            ctypes.memmove(hits.ctypes.data, hp.value, nh.value * 4)
        if release:
            _check(lib().mb_serve_release(self._h, ticket), "mb_serve_release")
        return sm, hits, lat.value

    def stats(self):
        sl, g, m = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().mb_serve_stats(self._h, ctypes.byref(sl), ctypes.byref(g), ctypes.byref(m)),
               "mb_serve_stats")
        return dict(slots=sl.value, groups=g.value, merged=m.value)

    COUNTERS = ("slots", "groups", "merged", "slots_created", "slots_released", "alloc_failures",
                "outgrown_groups", "busy", "memory_wait_ms", "slot_bytes", "reserve_bytes", "long_groups",
                "worker_busy_ms")

    def counters(self):
        v = np.zeros(len(self.COUNTERS), dtype=np.uint64)
        _check(lib().mb_serve_counters(self._h, _ptr(v), len(v)), "mb_serve_counters")
        return dict(zip(self.COUNTERS, (int(x) for x in v)))

    def inject(self, free_bytes: int = -1, fail_slots: int = 0):
        """Admission fault injection (tests): fake free device memory, failing slot creations."""
        _check(lib().mb_serve_inject(self._h, free_bytes, fail_slots), "mb_serve_inject")

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().mb_serve_destroy(self._h), "mb_serve_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_l2_fetch_granularity(nbytes: int = 32) -> int:
    """cudaLimitMaxL2FetchGranularity of this process's context (0 = query); returns the value
    in force."""
    now = ctypes.c_int()
    _check(lib().mb_set_l2_fetch_granularity(nbytes, ctypes.byref(now)), "mb_set_l2_fetch_granularity")
    return now.value
