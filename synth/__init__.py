"""Seeded synthetic inputs (reference genomes and reads) for the seeding stage.

Shared by the CPU oracle and the GPU path; holds none of the method's
arithmetic.  The generator is plain C (``synth.c``), compiled on first use with
gcc, and draws the same bytes on x86 and Arm hosts.

The workload recipes follow the paper's evaluation inputs (2x150 bp
paired-end WGS reads and mixed short/long reads, Section 3.1), which are not
available here; seeded i.i.d. and repeat-structured genomes stand in for
GRCh38.  Base codes: 0=A 1=C 2=G 3=T 4=N.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

# seeds of the five workloads: 0x6D62000i
SEED = {i: 0x6D620000 + i for i in range(1, 6)}


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libsynth.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                           src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


class _ReadOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("read_len", ctypes.c_uint32),
                ("len_lo", ctypes.c_uint32), ("len_hi", ctypes.c_uint32),
                ("sub_lo", ctypes.c_double), ("sub_hi", ctypes.c_double),
                ("indel", ctypes.c_double), ("frag_mean", ctypes.c_double),
                ("frag_sd", ctypes.c_double), ("bisulfite", ctypes.c_int),
                ("bs_noncpg", ctypes.c_double), ("bs_cpg", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.synth_ref.argtypes = [P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.synth_ref.restype = None
            L.synth_read_lengths.argtypes = [ctypes.POINTER(_ReadOpts), ctypes.c_uint64,
                                             ctypes.c_uint32, P]
            L.synth_read_lengths.restype = ctypes.c_uint64
            L.synth_reads.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(_ReadOpts), ctypes.c_uint64,
                                      ctypes.c_uint32, P, P, P]
            L.synth_reads.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def reference(length: int, seed: int, tandem: float = 0.0, segdup: float = 0.0,
              satellite: float = 0.0, nrun: float = 0.0) -> np.ndarray:
    """A reference of `length` bases (uint8 codes, 4 = N)."""
    out = np.empty(length, dtype=np.uint8)
    lib().synth_ref(_ptr(out), length, seed, tandem, segdup, satellite, nrun)
    return out


@dataclass
class Reads:
    seq: np.ndarray      # uint8 codes, reads concatenated
    off: np.ndarray      # uint64, n_reads + 1 offsets into seq
    origin: np.ndarray   # uint64, template start on the forward strand | strand << 63
    mate: np.ndarray     # uint8: 0 single-end, 1 read 1, 2 read 2

    @property
    def n(self) -> int:
        return len(self.off) - 1

    def read(self, i: int) -> np.ndarray:
        return self.seq[self.off[i]:self.off[i + 1]]

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        lens = (self.off[idx + 1] - self.off[idx]).astype(np.uint64)
        off = np.zeros(len(idx) + 1, dtype=np.uint64)
        np.cumsum(lens, out=off[1:])
        seq = np.concatenate([self.read(int(i)) for i in idx]) if len(idx) else np.zeros(0, np.uint8)
        return Reads(seq.astype(np.uint8), off, self.origin[idx].copy(), self.mate[idx].copy())


def reads(ref: np.ndarray, n_reads: int, seed: int, *, mode: int = 0, read_len: int = 150,
          len_lo: int = 100, len_hi: int = 10000, sub_lo: float = 0.0, sub_hi: float | None = None,
          indel: float = 0.0, frag_mean: float = 400.0, frag_sd: float = 50.0,
          bisulfite: bool = False, bs_noncpg: float = 0.98, bs_cpg: float = 0.30) -> Reads:
    """Reads sampled from both strands of `ref`.

    mode 0: single-end, fixed length; mode 1: paired-end (reads 2i, 2i+1 are
    mates, n_reads must be even); mode 2: single-end, log-uniform length in
    [len_lo, len_hi].  Substitution rate ramps from sub_lo at the first base to
    sub_hi at the last; indels are 1-3 bp at `indel` per base.
    """
    if mode == 1 and n_reads % 2:
        raise ValueError("paired-end read count must be even")
    o = _ReadOpts(mode, read_len, len_lo, len_hi, sub_lo, sub_lo if sub_hi is None else sub_hi,
                  indel, frag_mean, frag_sd, int(bisulfite), bs_noncpg, bs_cpg)
    off = np.empty(n_reads + 1, dtype=np.uint64)
    total = lib().synth_read_lengths(ctypes.byref(o), seed, n_reads, _ptr(off))
    seq = np.empty(total, dtype=np.uint8)
    origin = np.empty(n_reads, dtype=np.uint64)
    lib().synth_reads(_ptr(ref), len(ref), ctypes.byref(o), seed, n_reads, _ptr(off), _ptr(seq),
                      _ptr(origin))
    if mode == 1:
        mate = np.tile(np.array([1, 2], dtype=np.uint8), n_reads // 2)
    else:
        mate = np.zeros(n_reads, dtype=np.uint8)
    return Reads(seq, off, origin, mate)


# ----------------------------------------------------------------------------------------------
# Workload recipes.  `scale` shrinks the reference and the read count together for tests.

def repeat_rich_reference(length: int, seed: int, repeat_frac: float = 0.08) -> np.ndarray:
    """Uniform ACGT with tandem : segmental-duplication : satellite repeats in the
    ratio 5 : 2 : 1 covering `repeat_frac` of the sequence, plus 0.5% N runs."""
    return reference(length, seed, tandem=repeat_frac * 5 / 8, segdup=repeat_frac * 2 / 8,
                     satellite=repeat_frac * 1 / 8, nrun=0.005)


def workload(cfg: int, scale: float = 1.0, bisulfite: bool = False):
    """Return (ref, reads, params) of workload `cfg` (1..4) at `scale`.

    1: 1 Mbp uniform reference, 10,000 single-end 150 bp reads, 0.5% substitutions.
    2: 100 Mbp reference (8% repeats, 0.5% N), 1M 2x150 bp pairs, insert N(400,50),
       substitutions ramping 0.1% -> 1% along the read, 0.01% 1-3 bp indels.
    3: 1 Gbp reference (45% repeats), 10M pairs as in 2; `bisulfite` gives the
       directional bisulfite read set (1M pairs, 98% non-CpG / 30% CpG conversion).
    4: the 100 Mbp reference of 2, 200,000 single-end reads of log-uniform length
       100 bp - 10 kb, 0.1% substitutions, 0.02% indels.
    """
    params = dict(min_len=19, min_occ=1, max_occ=500, sa_rate=32)
    if cfg == 1:
        ref = reference(max(int(1_000_000 * scale), 2000), SEED[1])
        rd = reads(ref, max(int(10_000 * scale), 16), SEED[1] + 100, mode=0, read_len=150,
                   sub_lo=0.005)
    elif cfg in (2, 4):
        ref = repeat_rich_reference(max(int(100_000_000 * scale), 20000), SEED[2], 0.08)
        if cfg == 2:
            n = max(int(1_000_000 * scale), 8) * 2
            rd = reads(ref, n, SEED[2] + 100, mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01,
                       indel=0.0001)
        else:
            rd = reads(ref, max(int(200_000 * scale), 8), SEED[4] + 100, mode=2, len_lo=100,
                       len_hi=10000, sub_lo=0.001, indel=0.0002)
    elif cfg == 3:
        ref = repeat_rich_reference(max(int(1_000_000_000 * scale), 20000), SEED[3], 0.45)
        if bisulfite:
            rd = bisulfite_reads(ref, scale)
        else:
            n = max(int(10_000_000 * scale), 8) * 2
            rd = reads(ref, n, SEED[3] + 100, mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01,
                       indel=0.0001)
    else:
        raise ValueError(cfg)
    return ref, rd, params


def bisulfite_reads(ref: np.ndarray, scale: float = 1.0) -> Reads:
    """The directional bisulfite read set of workload 3 on `ref`: 1M pairs (x scale) of 2x150 bp,
    read 1 C->T and read 2 G->A at 98% of non-CpG and 30% of CpG C, substitutions and indels as in
    workload 3."""
    n = max(int(1_000_000 * scale), 8) * 2
    return reads(ref, n, SEED[3] + 200, mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01, indel=0.0001,
                 bisulfite=True)


def rescue_pairs(ref: np.ndarray, n_pairs: int, seed: int, read_len: int = 150, win_len: int = 600,
                 true_frac: float = 0.5, sub: float = 0.01):
    """(read, reference window) pairs shaped like mate rescue: a window of `win_len` bases at a
    uniform place of `ref`; for a `true_frac` share of pairs the read is a `read_len` substring
    of the window (substitutions at rate `sub`), otherwise it comes from a uniform place
    elsewhere; each pair is reverse-complemented as a whole with probability 1/2.
    Returns (reads, read_off, wins, win_off), bases as codes 0..3 (4 = N, from the reference)."""
    rng = np.random.default_rng(seed)
    L = len(ref)
    comp = np.array([3, 2, 1, 0, 4], dtype=np.uint8)
    reads_out = np.empty(n_pairs * read_len, np.uint8)
    wins_out = np.empty(n_pairs * win_len, np.uint8)
    step = 65536
    for a in range(0, n_pairs, step):
        k = min(step, n_pairs - a)
        w0 = rng.integers(0, L - win_len, k)
        x = rng.integers(0, win_len - read_len + 1, k)
        other = rng.integers(0, L - read_len, k)
        is_true = rng.random(k) < true_frac
        flip = rng.random(k) < 0.5
        W = ref[w0[:, None] + np.arange(win_len)[None, :]]
        R = ref[np.where(is_true, w0 + x, other)[:, None] + np.arange(read_len)[None, :]]
        mut = rng.random(R.shape) < sub
        R = np.where(mut & (R < 4), (R + rng.integers(1, 4, R.shape)) % 4, R).astype(np.uint8)
        W[flip] = comp[np.minimum(W[flip], 4)][:, ::-1]
        R[flip] = comp[np.minimum(R[flip], 4)][:, ::-1]
        reads_out[a * read_len:(a + k) * read_len] = R.reshape(-1)
        wins_out[a * win_len:(a + k) * win_len] = W.reshape(-1)
    roff = np.arange(n_pairs + 1, dtype=np.uint64) * read_len
    woff = np.arange(n_pairs + 1, dtype=np.uint64) * win_len
    return reads_out, roff, wins_out, woff


def planted_copies(unit_len: int, copies, spacer: int, seed: int):
    """A reference holding copies[u] exact copies of random unit u (`unit_len` bases each, one
    unit per entry of `copies`), in random order, separated (and flanked) by random spacers of
    `spacer` bases, all bases drawn uniformly (numpy, seeded).  Returns (reference, units, starts): units[u] is the u-th unit's bases and
    starts[u] the sorted reference positions of its copies.  With long random units and spacers
    no unit occurs anywhere else, or on the other strand, except with negligible probability, so a
    read equal to unit u occurs exactly copies[u] times in R . revcomp(R)."""
    rng = np.random.default_rng(seed)
    n_units = len(copies)
    units = rng.integers(0, 4, (n_units, unit_len)).astype(np.uint8)
    order = rng.permutation(np.repeat(np.arange(n_units), copies))
    parts, starts, pos = [], [[] for _ in range(n_units)], 0
    for u in order:
        sp = rng.integers(0, 4, spacer).astype(np.uint8)
        parts.append(sp)
        pos += spacer
        starts[u].append(pos)
        parts.append(units[u])
        pos += unit_len
    parts.append(rng.integers(0, 4, spacer).astype(np.uint8))
    return np.concatenate(parts), units, [np.array(s, dtype=np.uint64) for s in starts]


def junction_read(ref_len: int, half: int, seed: int, filler_len: int = 0):
    """A reference whose first `half` bases are A/T only, and a 2*half-base read that ends with the
    reference's last `half` bases and continues with its first `half` bases.  Under the bisulfite
    conversion of read 1 (C -> T) the read spells the text across the boundary between the
    C-to-T copy and the G-to-A copy of the 3-base text CT(R) GA(R) ..., so its one occurrence
    spans two copies.  Returns (reference, read)."""
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 4, ref_len).astype(np.uint8)
    ref[:half] = np.where(rng.random(half) < 0.5, 0, 3).astype(np.uint8)
    read = np.concatenate([ref[ref_len - half:], ref[:half]]).astype(np.uint8)
    return ref, read
