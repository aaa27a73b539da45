"""CPU oracle of the seeding stage (SMEM finding, max-occurrence filter, locate).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  It shares
no code with the CUDA library (``paper_2606_15357_gb300``) and never imports
it.  The arithmetic lives in ``oracle.cpp`` (plain C++, compiled with g++ on
first use); this module only marshals numpy arrays.

What each function follows (arxiv 2606.15357):
  Index            Section 2.1: T = R . revcomp(R) . $, suffix array S, B[i] = T[S(i)-1];
                   Section 2.9: bisulfite mode indexes CT(R) . GA(R).
  ds_interval      Section 2.1, the ds-interval (lo(P), lo(revcomp P), occ(P)) by binary
                   search over the sorted suffixes.
  pi / backward_ext / forward_ext
                   Section 2.1 LF-mapping and Algorithm 1.
  smem(method="def")   Section 2.1 definition of (l,c)-SMEMs (the published answer).
  smem(method="alg3")  Algorithm 3 BatchFindSMEM with one FIFO queue.
  smem_brute       the definition by scanning T (tiny texts only).
  locate           {S(x) : k <= x < k+s} from the full suffix array (Section 2.4).
  locate_slow / batch_locate   Algorithm 2 with the sampled suffix array, modulo n.
  seed             the whole stage: SMEMs, max-occ filter, hits in SA-row order.

Parity pins (tests/test_oracle_*.py): brute force on tiny texts, the suffix
array as a sorted permutation, hand-derived values for short texts, closed
forms (empty pattern, N), invariants (non-containment, maximality, strand
mirror, hit positions spell the SMEM), Algorithm 3 = definition,
LocateSlow = BatchLocate = full suffix array.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

SMEM_DTYPE = np.dtype([("read", np.uint64), ("qbeg", np.uint64), ("qend", np.uint64),
                       ("k", np.uint64), ("kr", np.uint64), ("s", np.uint64)])


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (g++, OpenMP)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", src,
                           "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, U64, U32, U8, I = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint8, ctypes.c_int)
            sig = {
                "orc_index_build": ([P, U64, U64, I, U32, I], P),
                "orc_index_free": ([P], None),
                "orc_n": ([P], U64), "orc_rlen": ([P], U64), "orc_primary": ([P], U64),
                "orc_C": ([P, P], None), "orc_text": ([P, P], None), "orc_sa": ([P, P], None),
                "orc_bwt": ([P, P], None), "orc_ssa": ([P, P], None),
                "orc_pi": ([P, U8, U64], U64),
                "orc_ds_def": ([P, P, U64, P], None),
                "orc_ds_def_batch": ([P, P, U64, U64, P, I], None),
                "orc_backward_ext": ([P, P, U8, P], None),
                "orc_forward_ext": ([P, P, U8, P], None),
                "orc_smem": ([P, P, P, U32, U32, U32, I, I], P),
                "orc_smem_brute": ([P, U64, P, P, U32, U32, U32, I], P),
                "orc_result_nsmem": ([P], U64), "orc_result_smem": ([P, P], None),
                "orc_result_free": ([P], None),
                "orc_locate_sa": ([P, P, U64, P, I], None),
                "orc_locate_slow": ([P, P, U64, P, I], None),
                "orc_batch_locate": ([P, P, U64, P], None),
                "orc_count_alg3": ([P, P, P, U32, U32, U32, U64, U32, P], None),
                "orc_count_locate_join": ([P, P, U64, U32, P, I], None),
                "orc_count_locate": ([P, P, U64, P, I], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _take_smem(h) -> np.ndarray:
    L = lib()
    m = L.orc_result_nsmem(h)
    raw = np.empty(6 * m, dtype=np.uint64)
    if m:
        L.orc_result_smem(h, _p(raw))
    L.orc_result_free(h)
    return raw.view(SMEM_DTYPE).reshape(m)


class Index:
    """FMD-index of R (Section 2.1) built on the host by sorting suffixes."""

    def __init__(self, ref: np.ndarray, n_seed: int = 0, bs3: bool = False, sa_rate: int = 32,
                 threads: int = 0):
        self._ref = _u8(ref)
        self.sa_rate = sa_rate
        self.bs3 = bs3
        self._h = lib().orc_index_build(_p(self._ref), len(self._ref), n_seed, int(bs3), sa_rate,
                                        threads)
        self.n = int(lib().orc_n(self._h))
        self.rlen = int(lib().orc_rlen(self._h))
        self.primary = int(lib().orc_primary(self._h))
        C = np.empty(5, dtype=np.uint64)
        lib().orc_C(self._h, _p(C))
        self.C = C

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_index_free(h)
            self._h = None

    # raw arrays (oracle coding: $=0, A=1, C=2, G=3, T=4)
    def text(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.uint8)
        lib().orc_text(self._h, _p(out))
        return out

    def sa(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.uint32)
        lib().orc_sa(self._h, _p(out))
        return out

    def bwt(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.uint8)
        lib().orc_bwt(self._h, _p(out))
        return out

    def ssa(self) -> np.ndarray:
        out = np.empty((self.n + self.sa_rate - 1) // self.sa_rate, dtype=np.uint32)
        lib().orc_ssa(self._h, _p(out))
        return out

    def pi(self, a: int, k: int) -> int:
        """pi(a,k) with a in oracle coding (0 = $)."""
        return int(lib().orc_pi(self._h, a, k))

    def ds_interval(self, P) -> tuple:
        """ds-interval of P (read codes 0..3, 4 = N) by the definition."""
        P = _u8(P)
        out = np.empty(3, dtype=np.uint64)
        lib().orc_ds_def(self._h, _p(P), len(P), _p(out))
        return tuple(int(v) for v in out)

    def ds_intervals(self, pats: np.ndarray, threads: int = 0) -> np.ndarray:
        """ds-intervals of the rows of a 2-D uint8 array of patterns; shape (npat, 3)."""
        pats = np.ascontiguousarray(pats, dtype=np.uint8)
        out = np.empty((pats.shape[0], 3), dtype=np.uint64)
        if pats.shape[0]:
            lib().orc_ds_def_batch(self._h, _p(pats), pats.shape[0], pats.shape[1], _p(out), threads)
        return out

    def backward_ext(self, iv, a: int) -> tuple:
        inp = np.asarray(iv, dtype=np.uint64)
        out = np.empty(3, dtype=np.uint64)
        lib().orc_backward_ext(self._h, _p(inp), a, _p(out))
        return tuple(int(v) for v in out)

    def forward_ext(self, iv, a: int) -> tuple:
        inp = np.asarray(iv, dtype=np.uint64)
        out = np.empty(3, dtype=np.uint64)
        lib().orc_forward_ext(self._h, _p(inp), a, _p(out))
        return tuple(int(v) for v in out)

    def smem(self, seq, off, min_len: int = 19, min_occ: int = 1, method: str = "def",
             threads: int = 0) -> np.ndarray:
        seq, off = _u8(seq), _u64(off)
        h = lib().orc_smem(self._h, _p(seq), _p(off), len(off) - 1, min_len, min_occ,
                           {"def": 0, "alg3": 1, "alg3_cache": 2}[method], threads)
        return _take_smem(h)

    def locate(self, rows, threads: int = 0) -> np.ndarray:
        rows = _u64(rows)
        out = np.empty(len(rows), dtype=np.uint64)
        if len(rows):
            lib().orc_locate_sa(self._h, _p(rows), len(rows), _p(out), threads)
        return out

    def locate_slow(self, rows, threads: int = 0) -> np.ndarray:
        rows = _u64(rows)
        out = np.empty(len(rows), dtype=np.uint64)
        if len(rows):
            lib().orc_locate_slow(self._h, _p(rows), len(rows), _p(out), threads)
        return out

    def batch_locate(self, rows) -> np.ndarray:
        rows = _u64(rows)
        out = np.empty(len(rows), dtype=np.uint64)
        if len(rows):
            lib().orc_batch_locate(self._h, _p(rows), len(rows), _p(out))
        return out

    def count_alg3(self, seq, off, min_len: int = 19, min_occ: int = 1, block_rows: int = 64,
                   kmer_k: int = 0):
        """Work of Algorithm 3 over the reads: (extension steps with a base, blocks of
        `block_rows` rows those steps read: 1 if rows p and p+s share a block, else 2).  With
        kmer_k > 0 the steps are those Algorithm 3 takes with the ds-interval cache of all
        kmer_k-mers (Section 2.5), and a third value counts the cache lookups."""
        seq, off = _u8(seq), _u64(off)
        out = np.zeros(3, dtype=np.uint64)
        lib().orc_count_alg3(self._h, _p(seq), _p(off), len(off) - 1, min_len, min_occ, block_rows, kmer_k,
                             _p(out))
        if kmer_k:
            return int(out[0]), int(out[1]), int(out[2])
        return int(out[0]), int(out[1])

    def count_locate(self, rows, threads: int = 0) -> tuple:
        """Work of Algorithm 2 over the rows, the $ row counting as sampled with S = 0:
        (LF steps, sampled-S reads)."""
        rows = _u64(rows)
        out = np.zeros(2, dtype=np.uint64)
        if len(rows):
            lib().orc_count_locate(self._h, _p(rows), len(rows), _p(out), threads)
        return int(out[0]), int(out[1])

    def count_locate_join(self, rows, pass_bits: int = 3, threads: int = 0) -> tuple:
        """Work of locate with walks that join over the distinct rows in 2**pass_bits passes:
        (LF steps, sampled-S reads, walks stopped at a row of an earlier pass)."""
        rows = _u64(rows)
        out = np.zeros(3, dtype=np.uint64)
        if len(rows):
            lib().orc_count_locate_join(self._h, _p(rows), len(rows), pass_bits, _p(out), threads)
        return tuple(int(v) for v in out)

    def seed(self, seq, off, min_len: int = 19, min_occ: int = 1, max_occ: int = 500,
             threads: int = 0, method: str = "def"):
        """The whole seeding stage.  Returns (smem, over, hit_off, hits):
        over[m] = s > max_occ (not located); hit_off = exclusive prefix sum of
        the located hit counts; hits = S(x) for x in [k, k+s) of each kept SMEM,
        in SMEM order then SA-row order."""
        sm = self.smem(seq, off, min_len, min_occ, method, threads)
        over = sm["s"] > max_occ
        cnt = np.where(over, 0, sm["s"]).astype(np.uint64)
        hit_off = np.zeros(len(sm), dtype=np.uint64)
        if len(sm):
            np.cumsum(cnt[:-1], out=hit_off[1:])
        total = int(cnt.sum())
        rows = np.empty(total, dtype=np.uint64)
        keep = np.nonzero(~over)[0]
        for q in keep:
            b = int(hit_off[q])
            rows[b:b + int(cnt[q])] = np.arange(int(sm["k"][q]), int(sm["k"][q] + cnt[q]),
                                                dtype=np.uint64)
        hits = self.locate(rows, threads)
        return sm, over, hit_off, hits


def reseed(X: "Index", seq, off, first, min_len: int = 19, max_s: int = 10, max_occ: int = 500,
           threads: int = 0):
    """Section 2.6, second seeding round: for every first-round record with qend - qbeg >= 2l,
    s <= 10 and s <= max_occ, the (floor((qend - qbeg)/2), s + 1)-SMEMs of read[qbeg, qend) as a
    query of its own, by the definition (Index.smem).  Returns (records in read coordinates,
    ordered by window then qbeg; over-max-occ flags; hit offsets; hits)."""
    seq = _u8(seq)
    off = _u64(off)
    wins = [(int(x["read"]), int(x["qbeg"]), int(x["qend"]), int(x["s"])) for x in first
            if int(x["qend"]) - int(x["qbeg"]) >= 2 * min_len and int(x["s"]) <= max_s
            and int(x["s"]) <= max_occ]
    groups = {}
    for w, (r, b, e, s) in enumerate(wins):
        groups.setdefault(((e - b) // 2, s + 1), []).append(w)
    per_win = [[] for _ in wins]
    for (l2, c2), ws in groups.items():
        sub = np.concatenate([seq[int(off[wins[w][0]]) + wins[w][1]:int(off[wins[w][0]]) + wins[w][2]]
                              for w in ws])
        so = np.zeros(len(ws) + 1, dtype=np.uint64)
        np.cumsum([wins[w][2] - wins[w][1] for w in ws], out=so[1:])
        rec = X.smem(sub, so, l2, c2, "def", threads)
        for x in rec:
            w = ws[int(x["read"])]
            per_win[w].append((wins[w][0], int(x["qbeg"]) + wins[w][1], int(x["qend"]) + wins[w][1],
                               int(x["k"]), int(x["kr"]), int(x["s"])))
    flat = [t for lst in per_win for t in lst]
    sm = np.array(flat, dtype=np.uint64).reshape(-1, 6).view(SMEM_DTYPE).reshape(-1) if flat else \
        np.zeros(0, dtype=SMEM_DTYPE)
    over = sm["s"] > max_occ
    cnt = np.where(over, 0, sm["s"]).astype(np.uint64)
    hoff = np.zeros(len(sm), dtype=np.uint64)
    if len(sm):
        np.cumsum(cnt[:-1], out=hoff[1:])
    rows = np.concatenate([np.arange(int(x["k"]), int(x["k"]) + int(c), dtype=np.uint64)
                           for x, c in zip(sm, cnt)]) if len(sm) else np.zeros(0, np.uint64)
    return sm, over, hoff, X.locate(rows, threads)


def smem_brute(text: np.ndarray, seq, off, min_len: int = 19, min_occ: int = 1,
               threads: int = 0) -> np.ndarray:
    """(l,c)-SMEMs and their ds-intervals by scanning the text (oracle coding, ends with $)."""
    text, seq, off = _u8(text), _u8(seq), _u64(off)
    h = lib().orc_smem_brute(_p(text), len(text), _p(seq), _p(off), len(off) - 1, min_len,
                             min_occ, threads)
    return _take_smem(h)


def bs_convert_reads(seq, off, mate) -> np.ndarray:
    """Section 2.9: every C of read 1 becomes T and every G of read 2 becomes A."""
    seq = np.array(seq, dtype=np.uint8, copy=True)
    rid = np.repeat(np.arange(len(off) - 1), np.diff(np.asarray(off, dtype=np.int64)))
    m = np.asarray(mate)[rid]
    seq[(m == 1) & (seq == 1)] = 3
    seq[(m == 2) & (seq == 2)] = 0
    return seq


def bs_keep(pos, qlen, read_mate, rlen: int) -> np.ndarray:
    """Section 2.9 strand filter on the 3-base index T = CT(R) GA(R) rc(GA(R)) rc(CT(R)) $:
    a read-1 hit is kept only inside the forward C-to-T or the reverse G-to-A copy, a read-2
    hit only inside the forward G-to-A or the reverse C-to-T copy.  rlen = |R|; a hit that
    crosses a copy boundary is dropped."""
    pos = np.asarray(pos, dtype=np.int64)
    qlen = np.asarray(qlen, dtype=np.int64)
    seg = pos // rlen
    whole = (pos + qlen - 1) // rlen == seg
    m = np.asarray(read_mate)
    ok1 = (seg == 0) | (seg == 2)
    ok2 = (seg == 1) | (seg == 3)
    return whole & np.where(m == 1, ok1, np.where(m == 2, ok2, True))


PIECE_DTYPE = np.dtype([("hit", np.uint64), ("read", np.uint32), ("qbeg", np.uint32),
                        ("qend", np.uint32), ("pos", np.uint32)])


def bs_split(ref, seq, off, mate, sm, hits, keep, min_len: int = 19, over=None) -> np.ndarray:
    """Section 2.9, T-to-C split of bisulfite seed matches.  For every kept hit (record m of
    `sm`, text position p = hits[h]) the original read bases x_t = read[qbeg + t] are compared
    with the original reference bases under the seed: copy g = p // |R| of the 3-base text, offset
    q = p - g |R|; copies 0 and 1 read R[q + t], copies 2 and 3 (reverse complements) read
    comp(R[|R| - 1 - (q + t)]).  A read-1 seed (C->T converted) breaks where the read has C over a
    reference T; a read-2 seed (G->A) where the read has G over a reference A; other reads do not
    break.  The seed is cut at every such position (the position itself leaves the seed) and the
    pieces of at least min_len bases are returned as (hit, read, qbeg, qend, pos), pos = the
    piece's text position, in hit order then qbeg order.  `over` marks the records over max_occ
    (no hits); by default bit 0 of sm["flags"]."""
    ref = np.asarray(ref, dtype=np.uint8)
    seq = np.asarray(seq, dtype=np.uint8)
    off = np.asarray(off, dtype=np.int64)
    mate = np.asarray(mate)
    M = len(ref)
    comp = np.array([3, 2, 1, 0, 4], dtype=np.uint8)
    if over is None:   # records with a flags field (the library's layout): bit 0 = over max_occ
        over = (sm["flags"] & 1).astype(bool)
    cnt = np.where(over, 0, sm["s"]).astype(np.int64)
    out = []
    h = 0
    for m in range(len(sm)):
        rd, qb, qe = int(sm["read"][m]), int(sm["qbeg"][m]), int(sm["qend"][m])
        for _ in range(int(cnt[m])):
            if keep is None or keep[h]:
                p = int(hits[h])
                g, q = p // M, p - (p // M) * M
                L = qe - qb
                if g < 2:
                    R = ref[q:q + L]
                else:
                    R = comp[np.minimum(ref[M - q - L:M - q][::-1], 4)]
                x = seq[off[rd] + qb:off[rd] + qe]
                mt = int(mate[rd])
                if mt == 1:
                    cut = (x == 1) & (R == 3)
                elif mt == 2:
                    cut = (x == 2) & (R == 0)
                else:
                    cut = np.zeros(L, dtype=bool)
                edges = [-1] + np.nonzero(cut)[0].tolist() + [L]
                for a, b in zip(edges[:-1], edges[1:]):
                    if b - (a + 1) >= min_len:
                        out.append((h, rd, qb + a + 1, qb + b, p + a + 1))
            h += 1
    arr = np.zeros(len(out), dtype=PIECE_DTYPE)
    for i, t in enumerate(out):
        arr[i] = t
    return arr


def qmer_diag_max(P, R, q: int = 7) -> int:
    """Mate-rescue prefilter (Section 2.7): M_t = |{(i, j) : P[i, i+q) = R[j, j+q), j - i = t}|
    over every q-mer start i of P and j of R, and the result max_t M_t (0 when no q-mer matches).
    A q-mer holding an N (code > 3) matches nothing.  Written as the definition: all pairs (i, j)
    compared, matches counted per diagonal t."""
    P = np.asarray(P, dtype=np.int64)
    R = np.asarray(R, dtype=np.int64)
    if len(P) < q or len(R) < q:
        return 0
    counts = {}
    for i in range(len(P) - q + 1):
        a = P[i:i + q]
        if np.any(a > 3):
            continue
        for j in range(len(R) - q + 1):
            b = R[j:j + q]
            if np.array_equal(a, b):
                counts[j - i] = counts.get(j - i, 0) + 1
    return max(counts.values()) if counts else 0


def qmer_diag_max_batch(reads, read_off, wins, win_off, q: int = 7) -> np.ndarray:
    """qmer_diag_max for every (read, window) pair, by q-mer codes (same definition, vectorised
    per pair: codes compared by broadcasting, matches binned by j - i)."""
    reads = np.asarray(reads, dtype=np.uint8)
    wins = np.asarray(wins, dtype=np.uint8)
    read_off = np.asarray(read_off, dtype=np.int64)
    win_off = np.asarray(win_off, dtype=np.int64)
    out = np.zeros(len(read_off) - 1, dtype=np.uint32)

    def codes(x):
        n = len(x) - q + 1
        if n <= 0:
            return np.zeros(0, np.int64)
        c = np.zeros(n, np.int64)
        bad = np.zeros(n, bool)
        for k in range(q):
            s = x[k:k + n].astype(np.int64)
            bad |= s > 3
            c = c * 4 + np.minimum(s, 3)
        c[bad] = -1
        return c

    for p in range(len(out)):
        a = codes(reads[read_off[p]:read_off[p + 1]])
        b = codes(wins[win_off[p]:win_off[p + 1]])
        if len(a) == 0 or len(b) == 0:
            continue
        eq = (a[:, None] == b[None, :]) & (a[:, None] >= 0)
        i, j = np.nonzero(eq)
        if len(i):
            out[p] = np.bincount(j - i + len(a)).max()
    return out
