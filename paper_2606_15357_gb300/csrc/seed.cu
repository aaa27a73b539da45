// Seeding on the GPU: (l,c)-SMEM finding (Section 2.5, Algorithm 3), the max-occurrence flag,
// and locate through the sampled suffix array (Section 2.4, Algorithm 2).
//
// SMEMs: one thread runs Algorithm 3's three-stage state machine for one read.  In Algorithm 3
// every read has exactly one entry in the queue at any time, so the per-read order of queue
// operations is the serial order below; the GPU's many resident warps take the place of the
// paper's queue-plus-prefetch as the way to keep many block reads in flight.  Every step that
// touches memory is one extension (Algorithm 1), i.e. two occurrence-block reads, so all lanes
// of a warp share the same memory instruction whatever stage they are in.
//
// Output: each read first writes its SMEMs into a private run of slots in scratch memory
// (off[r]/16 + 8r slots before it), a prefix sum over the per-read counts gives the final
// positions, and a gather writes the 48-byte records.  Reads with more SMEMs than slots are
// listed and recomputed straight into the final records.
#include <climits>
#include <vector>
#include "common.cuh"

DevIndex mb_dev_index(const mb_index *x);
int mb_index_device(const mb_index *x);
u32 mb_index_flags(const mb_index *x);

namespace {

// second seeding round (Section 2.6): windows are SMEMs occurring at most this many times
constexpr u32 RESEED_MAX_OCC = 10;

struct SlotRec {
    u32 qbeg, qend, k, kr, s;
    u32 pos;   // the text position of the one occurrence when the kernel found it, else NOPOS
};
constexpr u32 NOPOS = 0xFFFFFFFFu;   // no known position (and, in a row list given to k_locate, a row to skip)

// Scratch slots: a read of len bases owns len/16 + 8 slots (about 17 for 150 bases).
constexpr u64 SLOT_DIV = 16, SLOT_EXTRA = 8;
__host__ __device__ __forceinline__ u64 slots_before(u64 bases_before, u64 r) {
    return bases_before / SLOT_DIV + SLOT_EXTRA * r;
}
__host__ __device__ __forceinline__ u64 slots_total(u64 bases, u64 n_reads) {
    return bases / SLOT_DIV + SLOT_EXTRA * n_reads + SLOT_EXTRA;
}
__device__ __forceinline__ u64 slot_base(const u64 *off, u64 r) { return slots_before(off[r] - off[0], r); }

// Work counters of the measurement mode (MB_COUNT); compiled out otherwise.
template <bool ON>
struct Work {
    u64 steps = 0, blocks = 0, kmer = 0, lf = 0, sa = 0, uwalk = 0, usample = 0, utext = 0, joins = 0;
    __device__ __forceinline__ void ext(u64 p, u64 s) {
        if (ON) {
            ++steps;
            blocks += (p >> BLK_SHIFT) == ((p + s) >> BLK_SHIFT) ? 1 : 2;
        }
    }
    __device__ __forceinline__ void flush(u64 *wc) {
        if (ON) {
            if (steps) atomicAdd((unsigned long long *)&wc[WC_EXT_STEPS], (unsigned long long)steps);
            if (blocks) atomicAdd((unsigned long long *)&wc[WC_EXT_BLOCKS], (unsigned long long)blocks);
            if (kmer) atomicAdd((unsigned long long *)&wc[WC_KMER], (unsigned long long)kmer);
            if (lf) atomicAdd((unsigned long long *)&wc[WC_LF_STEPS], (unsigned long long)lf);
            if (sa) atomicAdd((unsigned long long *)&wc[WC_SA_READS], (unsigned long long)sa);
            if (uwalk) atomicAdd((unsigned long long *)&wc[WC_U_WALK], (unsigned long long)uwalk);
            if (usample) atomicAdd((unsigned long long *)&wc[WC_U_SAMPLE], (unsigned long long)usample);
            if (utext) atomicAdd((unsigned long long *)&wc[WC_U_TEXT], (unsigned long long)utext);
            if (joins) atomicAdd((unsigned long long *)&wc[WC_JOINS], (unsigned long long)joins);
        }
    }
};

// Per-read state of Algorithm 3.  In Algorithm 3 a read has exactly one queue entry at any time,
// so one read's queue operations happen in the serial order kept here.
struct SmemState {
    const u8 *P;
    int lim;             // chunk loads must end by P + lim (the end of the batch, capped)
    int cj;              // P + cj is the 16-byte aligned start of the cached chunk (INT_MIN: none)
    uint4 chunk;         // the read's bases around the current position
    int L;       // read length
    u32 conv;    // bisulfite conversion (0 none, 1 C->T, 2 G->A)
    int u;       // stage 1, 2, 3; 0 = finished
    int i, j;
    u32 k, kr, s;
    bool tried;  // stage 3: the k-mer table was already consulted for this entry
    u32 pos;     // stages 5-6: text position of the one occurrence of P[i, j)
};

__device__ __forceinline__ void smem_begin(SmemState &S, const u8 *P, int L, u32 conv, u32 l, u32 n,
                                           const u8 *end) {
    S.P = P;
    const u64 room = (u64)(end - P);
    S.lim = room > 0x7FFFFFF0ull ? 0x7FFFFFF0 : (int)room;
    S.cj = INT_MIN;
    S.L = L;
    S.conv = conv;
    S.u = (int)l - 1 < L ? 1 : 0;   // Algorithm 3 queues a read only if l - 1 < |P|
    S.i = 0;
    S.j = (int)l - 1;
    S.k = 0; S.kr = 0; S.s = n;
    S.tried = false;
}

// Base j of the read through a one-chunk cache: the steps of Algorithm 3 move j by one, so the
// 16 bytes around j are loaded once per 16 steps instead of one byte per step (a byte load at
// the end of the batch, where a whole chunk would pass the buffer).
__device__ __forceinline__ u32 cached_base(SmemState &S, int j) {
    const int mis = (int)((uintptr_t)S.P & 15);   // P's offset inside its 16-byte chunk
    const int cj = ((j + mis) & ~15) - mis;       // read index at which j's chunk starts
    u32 b;
    if (cj != S.cj && cj + 16 <= S.lim) {
        S.chunk = __ldg(reinterpret_cast<const uint4 *>(S.P + cj));
        S.cj = cj;
    }
    if (cj == S.cj) {
        const u32 o = (u32)(j - cj);
        const u32 w = o < 8 ? (o < 4 ? S.chunk.x : S.chunk.y) : (o < 12 ? S.chunk.z : S.chunk.w);
        b = (w >> (8 * (o & 3))) & 0xFFu;
    } else {
        b = S.P[j];
    }
    if (S.conv == 1 && b == 1) b = 3;
    if (S.conv == 2 && b == 2) b = 0;
    return b;
}

// Eight bases (bytes 0..3) to their 2-bit codes, first base in the lowest bits (16 bits).
__device__ __forceinline__ u32 pack8(u64 x) {
    x = (x | (x >> 6)) & 0x000F000F000F000FULL;
    x = (x | (x >> 12)) & 0x000000FF000000FFULL;
    return (u32)((x | (x >> 24)) & 0xFFFFULL);
}
// Bisulfite conversion of eight bases at once (conv 1: C(1) -> T(3); conv 2: G(2) -> A(0)).
__device__ __forceinline__ u64 convert8(u64 x, u32 conv) {
    const u64 ONES = 0x0101010101010101ULL;
    if (conv == 1) return x | ((x & ~(x >> 1) & ONES) << 1);
    if (conv == 2) return x & ~((((x >> 1) & ~x) & ONES) << 1);
    return x;
}

// k-mer code of P[j-K+1 .. j] (K <= 16), first base in the lowest bits; false if it holds an N.
// The K bytes lie in two aligned 16-byte chunks: both are loaded, the K bytes shifted out, and
// tested, converted and packed eight at a time.  Next to the end of the batch it goes byte by
// byte.
__device__ __forceinline__ bool kmer_code(SmemState &S, int j, u32 K, u32 &code) {
    const int st = j - (int)K + 1;
    const u8 *a = S.P + st;
    const u8 *A = (const u8 *)((uintptr_t)a & ~(uintptr_t)15);
    const u32 o = (u32)(a - A);
    if ((long long)(A + 32 - S.P) <= (long long)S.lim) {
        const ulonglong2 c0 = __ldg(reinterpret_cast<const ulonglong2 *>(A));
        const ulonglong2 c1 = __ldg(reinterpret_cast<const ulonglong2 *>(A + 16));
        const u64 w0 = o < 8 ? c0.x : c0.y, w1 = o < 8 ? c0.y : c1.x, w2 = o < 8 ? c1.x : c1.y;
        const u32 sh = 8 * (o & 7);
        u64 lo = sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
        u64 hi = sh ? (w1 >> sh) | (w2 << (64 - sh)) : w1;
        lo &= K >= 8 ? ~0ULL : ((1ULL << (8 * K)) - 1);
        hi &= K >= 16 ? ~0ULL : (K > 8 ? ((1ULL << (8 * (K - 8))) - 1) : 0ULL);
        if (((lo | hi) & 0xFCFCFCFCFCFCFCFCULL) != 0) return false;   // an N (any code > 3)
        code = pack8(convert8(lo, S.conv)) | (pack8(convert8(hi, S.conv)) << 16);
        return true;
    }
    u32 v = 0;
    for (u32 t = 0; t < K; ++t) {
        const u32 b = cached_base(S, st + (int)t);
        if (b > 3) return false;
        v |= b << (2 * t);
    }
    code = v;
    return true;
}

// Up to 16 read bases from P[j] on as 2-bit codes (first in the low bits, bisulfite conversion
// applied) with a mask of the N among them (bit 2t for base j + t); returns how many (at least 1).
// The 16-byte chunk holding j is loaded if it is not the cached one; next to the end of the batch
// it takes one base by a byte load.
__device__ __forceinline__ u64 byte_flags(u64 x) {   // bit 0 of each byte: the byte is above 3
    u64 t = x & 0xFCFCFCFCFCFCFCFCULL;
    t |= t >> 4;
    t |= t >> 2;
    t |= t >> 1;
    return t & 0x0101010101010101ULL;
}
__device__ __forceinline__ u32 read_codes16(SmemState &S, int j, u32 &codes, u32 &nmask) {
    const int mis = (int)((uintptr_t)S.P & 15);
    const int cj = ((j + mis) & ~15) - mis;
    if (cj != S.cj && cj + 16 <= S.lim) {
        S.chunk = __ldg(reinterpret_cast<const uint4 *>(S.P + cj));
        S.cj = cj;
    }
    if (cj == S.cj) {
        const u32 o = (u32)(j - cj);
        const u64 lo = ((u64)S.chunk.y << 32) | S.chunk.x, hi = ((u64)S.chunk.w << 32) | S.chunk.z;
        const u64 M3 = 0x0303030303030303ULL;
        const u32 nm = pack8(byte_flags(lo)) | (pack8(byte_flags(hi)) << 16);
        const u32 cd = pack8(convert8(lo & M3, S.conv)) | (pack8(convert8(hi & M3, S.conv)) << 16);
        codes = cd >> (2 * o);
        nmask = nm >> (2 * o);
        return 16 - o;
    }
    const u32 b = cached_base(S, j);
    codes = b & 3u;
    nmask = b > 3 ? 1u : 0u;
    return 1;
}

// What a lane does with memory in one step of Algorithm 3.
enum { ACT_NONE = 0, ACT_EXT = 1, ACT_KMER = 2, ACT_WALK = 3, ACT_SAMPLE = 4, ACT_TEXT = 5 };

// A match that occurs once (s = 1) in stage 2 can be extended forwards by comparing the read with
// the text after its one occurrence instead of one ForwardExt per base: P[i, j+1) occurs iff
// T[pos + j - i] = P[j], where pos is the occurrence of P[i, j), and while s = 1 the row k of
// P[i, j) stays the row of the suffix at pos.  Stages 4-7 do that, with the same result as
// Algorithm 3's steps (and the same transitions: emit, then stage 3 or the end of the read):
//   4  walk from row k to a row that is a multiple of AUX_RATE (or the $ row): pos = S(row) + steps
//      (kr holds the walking row, s the steps)
//   5  compare up to 16 bases of the read and the text per memory action
//   6  kr of the final match = the row of the suffix at y = n - 1 - pos - (j - i) (its reverse
//      complement's one occurrence): start from the ISA sample at the next multiple of AUX_RATE
//   7  walk back from there to y (s counts down), then emit (i, j, k, kr, 1)
// It is used when at least U_MIN bases of the read remain, where the walks cost less than the
// steps they replace.
constexpr int U_MIN = 16;

// The memory actions of the uniform step of k_smem_split: block reads (an extension or an LF step
// of a walk), a text comparison, an SA / ISA sample, a k-mer table entry.
enum { R_BLOCK = 0, R_TEXT = 1, R_SAMPLE = 2, R_KMER = 3 };

// Stages 4-7 up to their next memory action: R_BLOCK (a walk step), R_SAMPLE (sa_aux in stage 4,
// isa_aux in stage 6, index in acode) or R_TEXT.  Returns false only in stage 7 with the walk
// done (s = 0), where the match is emitted.
__device__ __forceinline__ bool uniq_next(SmemState &S, u32 n, u32 prim, int &ract, u32 &acode) {
    for (;;) {
        if (S.u == 4) {
            if (S.kr == prim) {                     // the $ row: S = 0
                S.pos = S.s;
                S.u = 5;
                continue;
            }
            if ((S.kr & (AUX_RATE - 1)) == 0) {
                acode = S.kr / AUX_RATE;
                ract = R_SAMPLE;
                return true;
            }
            if (S.s > n) {                          // only on a corrupted index: compare nothing
                S.pos = n;
                S.u = 5;
                continue;
            }
            ract = R_BLOCK;
            return true;
        }
        if (S.u == 5) {
            if (S.j >= S.L || (u64)S.pos + (u32)(S.j - S.i) >= (u64)n - 1) {
                S.u = 6;
                continue;
            }
            ract = R_TEXT;
            return true;
        }
        if (S.u == 6) {
            const u64 end = (u64)S.pos + (u32)(S.j - S.i);
            const u64 y = end < (u64)n - 1 ? (u64)n - 1 - end : 0;
            u64 q = (y + AUX_RATE - 1) / AUX_RATE * AUX_RATE;
            if (q >= (u64)n - 1) {                  // the $ suffix, row 0
                q = (u64)n - 1;
                S.kr = 0;
                S.s = (u32)(q - y);
                S.u = 7;
                continue;
            }
            S.s = (u32)(q - y);
            acode = (u32)(q / AUX_RATE);
            ract = R_SAMPLE;
            return true;
        }
        if (S.u == 7 && S.s != 0) {
            ract = R_BLOCK;
            return true;
        }
        return false;
    }
}

// Tuning of k_smem_split: memory steps between two service passes, and lanes out of the loop that
// call a service pass early (defaults; mb_opts.smem_burst / smem_wait override them).
struct SmemTuning {
    u32 burst, wait;
    u32 rpw;   // reads a warp holds at once (lanes 0 .. rpw-1), 1..32
};
constexpr u32 SMEM_BURST = 8, SMEM_WAIT = 8;

// Moves through the steps of Algorithm 3 that need no memory and picks the next memory action:
// ACT_EXT, an extension of P[j] (backward in stages 1 and 3, forward in stage 2); ACT_KMER, a
// k-mer table lookup (its code in `code`); ACT_NONE, the read is finished.  SMEMs found on the
// way go to emit.
//
// With the k-mer table (Section 2.5), the first K backward steps from the empty string are one
// table lookup: the table holds exactly the interval those K BackwardExt steps give.  In stage 1
// a failing k-mer P[x, x+K) restarts the scan at x+1, no further than Algorithm 3's own restart
// (every window starting at or before x contains that k-mer, so none is a match); in stage 3 the
// restart point must be exact, so a failing k-mer falls back to single steps.
template <class Emit>
__device__ __forceinline__ int smem_next(SmemState &S, const DevIndex &I, u32 l, bool kmer, Emit &emit, u32 &code,
                                         bool uext = false) {
    const u32 n = (u32)I.n, K = I.kmer_k;
    for (;;) {
        if (S.u == 2) {
            if (S.j == S.L) {                       // reached the end of P
                emit(S.i, S.j, S.k, S.kr, S.s);
                S.u = 0;
                return ACT_NONE;
            }
            if (uext && S.s == 1 && S.L - S.j >= U_MIN) {   // one occurrence: compare text
                S.u = 4;
                S.kr = S.k;
                S.s = 0;
                continue;
            }
            return ACT_EXT;
        }
        if (S.u >= 4) {                             // stages 4-7
            int ract = R_BLOCK;
            if (uniq_next(S, n, (u32)I.primary, ract, code))
                return ract == R_TEXT ? ACT_TEXT : (ract == R_SAMPLE ? ACT_SAMPLE : ACT_WALK);
            emit(S.i, S.j, S.k, S.kr, 1u, S.pos);   // stage 7 done: P[i, j) occurs once
            if (S.j == S.L) {
                S.u = 0;
                return ACT_NONE;
            }
            S.u = 3;                                // as after a failed ForwardExt
            S.k = 0; S.kr = 0; S.s = n;
            S.tried = false;
            continue;
        }
        if (S.u == 1) {
            if (S.j < S.i) {                        // P[i, i+l) is a match: stage 2
                S.u = 2;
                S.j = S.i + (int)l;
                continue;
            }
            if (kmer && l >= K && S.s == n && kmer_code(S, S.j, K, code)) return ACT_KMER;
            return ACT_EXT;
        }
        if (S.u == 3) {
            if (S.j <= S.i) {                       // back to stage 1 at the next start
                S.u = 1;
                S.i = S.j + 1;
                S.j = S.j + (int)l;
                S.k = 0; S.kr = 0; S.s = n;
                continue;
            }
            if (kmer && !S.tried && S.s == n && S.j - (int)K + 1 > S.i && kmer_code(S, S.j, K, code)) {
                S.tried = true;
                return ACT_KMER;
            }
            return ACT_EXT;
        }
        return ACT_NONE;
    }
}

// Applies a k-mer table entry (tk, tkr, ts) looked up in stage 1 or 3.  Returns false when the
// read is finished.
__device__ __forceinline__ bool smem_apply_kmer(SmemState &S, u32 tk, u32 tkr, u32 ts, u32 l, u32 c, u32 K) {
    if (ts >= c) {                                  // the K steps all succeed
        S.k = tk; S.kr = tkr; S.s = ts;
        S.j -= (int)K;
        return true;
    }
    if (S.u == 3) return true;                      // stage 3: step one base at a time instead
    const int x = S.j - (int)K + 1;                 // stage 1: restart after the k-mer's first base
    if (x + (int)l < S.L) {
        S.i = x + 1;
        S.j = x + (int)l;
        return true;
    }
    S.u = 0;
    return false;
}

// Applies the result (nk, nkr, ns) of the pending extension.  Returns false when the read is
// finished.
template <class Emit>
__device__ __forceinline__ bool smem_apply(SmemState &S, u32 nk, u32 nkr, u32 ns, u32 l, u32 c, u32 n, Emit &emit) {
    if (S.u == 2) {
        if (ns >= c) {
            ++S.j;
            S.k = nk; S.kr = nkr; S.s = ns;
        } else {                                    // SMEM ends before P[j]: stage 3
            emit(S.i, S.j, S.k, S.kr, S.s);
            S.u = 3;
            S.k = 0; S.kr = 0; S.s = n;
            S.tried = false;
        }
        return true;
    }
    if (ns >= c) {                                  // BackStep succeeded
        --S.j;
        S.k = nk; S.kr = nkr; S.s = ns;
        return true;
    }
    if (S.j + (int)l < S.L) {                       // BackStep failed: restart after P[j]
        S.u = 1;
        S.i = S.j + 1;
        S.j = S.j + (int)l;
        S.k = 0; S.kr = 0; S.s = n;
        return true;
    }
    S.u = 0;
    return false;
}

// The pending extension of P[j]: BackwardExt((k,kr,s), a) in stages 1/3, ForwardExt in stage 2
// (= BackwardExt((kr,k,s), comp a)).  The block reads are issued before the read base is fetched
// (the base is only needed for the counting), so their latencies overlap.  An N gives the empty
// interval.
template <class W>
__device__ __forceinline__ void smem_extend(SmemState &S, const DevIndex &I, u32 &nk, u32 &nkr, u32 &ns,
                                            W &work) {
    const bool fwd = S.u == 2;
    const u32 p = fwd ? S.kr : S.k, q = fwd ? S.k : S.kr, e = p + S.s;
    const Blk b0 = load_blk(I.occ + (p >> BLK_SHIFT));
    Blk b1 = b0;
    if ((e >> BLK_SHIFT) != (p >> BLK_SHIFT)) b1 = load_blk(I.occ + (e >> BLK_SHIFT));
    const u32 a = cached_base(S, S.j);
    nk = 0; nkr = 0; ns = 0;
    if (a < 4) {
        work.ext(p, S.s);
        const Ext x = extend_blocks(I, b0, b1, p, q, S.s, fwd ? 3u - a : a);
        nk = fwd ? x.q : x.p;
        nkr = fwd ? x.p : x.q;
        ns = x.s;
    }
}

// Algorithm 3 for one read, start to end (used by the overflow pass).
template <class Emit, class W>
__device__ __forceinline__ void smem_read(const DevIndex &I, const u8 *__restrict__ P, int L, u32 l, u32 c, u32 conv,
                                          bool kmer, const u8 *end, Emit &emit, W &work) {
    SmemState S;
    const u32 n = (u32)I.n;
    smem_begin(S, P, L, conv, l, n, end);
    for (;;) {
        u32 code = 0;
        const int act = smem_next(S, I, l, kmer, emit, code);
        if (act == ACT_NONE) break;
        if (act == ACT_KMER) {
            const u32 *t = I.kmer + 3 * (u64)code;
            work.kmer += 1;
            if (!smem_apply_kmer(S, __ldg(t), __ldg(t + 1), __ldg(t + 2), l, c, I.kmer_k)) break;
            continue;
        }
        u32 nk, nkr, ns;
        smem_extend(S, I, nk, nkr, ns, work);
        if (!smem_apply(S, nk, nkr, ns, l, c, n, emit)) break;
    }
}

struct SlotEmit {
    SlotRec *slots;
    u64 base;
    u32 cap, cnt;
    __device__ __forceinline__ void operator()(int i, int j, u32 k, u32 kr, u32 s, u32 pos = NOPOS) {
        if (cnt < cap) slots[base + cnt] = SlotRec{(u32)i, (u32)j, k, kr, s, pos};
        ++cnt;
    }
};

__device__ __forceinline__ u32 conv_of(const u8 *mate, u64 r, u32 bs) {
    if (!bs || !mate) return 0;
    u8 m = mate[r];
    return m == 1 ? 1u : (m == 2 ? 2u : 0u);
}

// Work distribution shared by the seeding kernels: each warp owns one contiguous range of items
// and hands the next item of its range to each lane that finishes, in lane order (ballot rank).
// The loop is warp-uniform: every iteration starts with all 32 lanes converged, so one memory
// instruction serves every lane that has work.
struct WarpRange {
    u64 next, end;
    __device__ __forceinline__ void init(u64 total) {
        const u64 gw = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5;
        const u64 nw = ((u64)gridDim.x * blockDim.x) >> 5;
        const u64 per = (total + nw - 1) / nw;
        next = gw * per < total ? gw * per : total;
        end = next + per < total ? next + per : total;
    }
};

// One lane keeps one read in flight; each loop iteration performs at most one extension per lane.
// QUEUE = false: reads are dealt out in warp ranges (WarpRange).  QUEUE = true: warps take the
// next reads from a device work queue (perm[*qhead ...], an atomic head), so long and short reads
// balance across the whole GPU in one launch.  A read whose slots would pass slot_total writes
// none (it is recomputed by the overflow pass).
struct SmemArgs {
    DevIndex I;
    const u8 *seq;
    const u64 *off;
    u32 nr;
    const u8 *mate;
    u32 bs, l, c;
    bool kmer;
    SlotRec *slots;
    u64 slot_total;
    u64 *counts;
    u32 *ovf_list, *ovf_n;
    const u32 *perm;
    u32 *qhead;
    u64 *wc;
    const u32 *lc;   // per-read (l | c << 16), or null for the kernel-wide l and c
    bool uext;       // extend matches that occur once by comparing text (stages 4-7)
    u32 *err = nullptr;                // device error word (always given)
    u32 *chk = nullptr;                // with MB_CHECKED: the error word, for the per-step bounds checks
    bool split = true;                 // k_smem_split (else k_smem, one loop for every stage)
    u32 warps = 0;                     // k_smem_split: resident warps per SM aimed at (0: by block size)
    SmemTuning tune = {SMEM_BURST, SMEM_WAIT, 32};
};

// Launch bounds per shape: 128 threads allow 85 registers (6 blocks, 24 warps per SM); 256 and
// 512 threads cap registers at 64 (32 warps per SM).
template <bool COUNT, bool QUEUE, int BLOCK>
__global__ void __launch_bounds__(BLOCK, BLOCK == 128 ? 6 : 1024 / BLOCK) k_smem(DevIndex I, const u8 *__restrict__ seq,
                                                               const u64 *__restrict__ off, u32 nr,
                                                               const u8 *__restrict__ mate, u32 bs, u32 l, u32 c,
                                                               bool kmer,
                                                               SlotRec *__restrict__ slots, u64 slot_total,
                                                               u64 *__restrict__ counts, u32 *__restrict__ ovf_list,
                                                               u32 *__restrict__ ovf_n, const u32 *__restrict__ perm,
                                                               u32 *qhead, u64 *wc, const u32 *__restrict__ lc,
                                                               bool uext, u32 *err) {
    const u32 lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    const u32 n = (u32)I.n;
    const u64 o0 = off[0];
    const u64 o1 = off[nr];
    const u8 *const end = seq + o1;
    Work<COUNT> work;
    SmemState S;
    SlotEmit em;
    WarpRange wr;
    if (!QUEUE) wr.init(nr);
    u32 lr = l, cr = c;   // this read's l and c
    auto start = [&](u64 rr) {
        u64 b = off[rr], e = off[rr + 1];
        bool bad = b > e || b < o0 || e > o1;
        if (bad) {   // offsets outside the batch or decreasing: nothing is read, no record written
            atomicOr(err, (u32)DEVCHK_OFFSETS);
            b = e = o0;
        }
        const u64 sb = slots_before(b - o0, rr), se = slots_before(e - o0, rr + 1);
        em.slots = slots;
        em.base = sb;
        em.cap = !bad && se <= slot_total ? (u32)(se - sb) : 0u;
        em.cnt = 0;
        if (lc) {
            const u32 v = lc[rr];
            lr = v & 0xFFFFu;
            cr = v >> 16;
        }
        smem_begin(S, seq + b, (int)(e - b), conv_of(mate, rr, bs), lr, n, end);
    };
    // next `k` items of this warp's work; lane gets item base + rank
    auto take = [&](u32 k, u32 rank, u64 &item, bool &ok) {
        if (QUEUE) {
            u32 base = 0;
            if (lane == 0) base = atomicAdd(qhead, k);
            base = __shfl_sync(0xffffffffu, base, 0);
            item = (u64)base + rank;
            ok = item < nr;
        } else {
            item = wr.next + rank;
            ok = item < wr.end;
            wr.next += k;
        }
    };
    u64 item, r = 0;
    bool live;
    take(32, lane, item, live);
    if (live) {
        r = QUEUE && perm ? perm[item] : item;
        start(r);
    }
    for (;;) {
        if (__all_sync(0xffffffffu, !live)) break;
        // phase 1 (divergent, no memory): stage changes, then this lane's one memory action
        int act = ACT_NONE;
        u32 code = 0;
        if (live) act = smem_next(S, I, lr, kmer && lr >= I.kmer_k, em, code, uext);
        __syncwarp();
        // phase 2 (converged): every lane's loads are issued before any is used, so the table
        // lookups, the block reads and the read-chunk reloads of one iteration overlap
        u32 tk = 0, tkr = 0, ts = 0;
        if (act == ACT_KMER) {
            const u32 *t = I.kmer + 3 * (u64)code;
            tk = __ldg(t);
            tkr = __ldg(t + 1);
            ts = __ldg(t + 2);
        }
        // an LF step of a walk (stages 4 and 7) is Algorithm 1's p' = C[a] + #a in B[0, p) with a = B[p]
        // and s = 0, so it shares the extension's loads and arithmetic
        const bool walk = act == ACT_WALK, fwd = S.u == 2;
        const u32 p = (fwd || walk) ? S.kr : S.k, q = fwd ? S.k : S.kr, sz = walk ? 0u : S.s, e = p + sz;
        Blk b0, b1;
        u32 smp = 0, t0 = 0, t1 = 0, rc = 0, rn = 0, rcnt = 0;
        if (act == ACT_EXT || walk) {
            b0 = load_blk(I.occ + (p >> BLK_SHIFT));
            b1 = b0;
            if ((e >> BLK_SHIFT) != (p >> BLK_SHIFT)) b1 = load_blk(I.occ + (e >> BLK_SHIFT));
        } else if (act == ACT_SAMPLE) {
            smp = __ldg((S.u == 4 ? I.sa_aux : I.isa_aux) + code);
        } else if (act == ACT_TEXT) {
            const u32 x = S.pos + (u32)(S.j - S.i);
            t0 = __ldg(I.text2 + (x >> 4));
            t1 = __ldg(I.text2 + (x >> 4) + 1);
            rcnt = read_codes16(S, S.j, rc, rn);
        }
        const u32 a = act == ACT_EXT ? cached_base(S, S.j) : 0u;
        // phase 3: apply the results
        bool fin = false;
        if (act == ACT_KMER) {
            work.kmer += 1;
            fin = !smem_apply_kmer(S, tk, tkr, ts, lr, cr, I.kmer_k);
        } else if (act == ACT_EXT || walk) {
            const u32 sym = walk ? sym_at(b0, p & BLK_MASK) : (fwd ? 3u - a : a);
            Ext x{0, 0, 0};
            if (walk || a < 4) x = extend_blocks(I, b0, b1, p, q, sz, sym);   // an N: the empty interval
            if (walk) {                       // stage 4 counts steps up, stage 7 down
                work.uwalk += 1;
                S.kr = x.p;
                S.s = S.u == 4 ? S.s + 1 : S.s - 1;
            } else {
                if (a < 4) work.ext(p, S.s);
                fin = !smem_apply(S, fwd ? x.q : x.p, fwd ? x.p : x.q, x.s, lr, cr, n, em);
            }
        } else if (act == ACT_SAMPLE) {
            work.usample += 1;
            if (S.u == 4) {
                S.pos = smp + S.s;
                S.u = 5;
            } else {
                S.kr = smp;
                S.u = 7;
            }
        } else if (act == ACT_TEXT) {         // the matching prefix of read and text
            work.utext += 1;
            const u32 x = S.pos + (u32)(S.j - S.i);
            const u32 tc = (u32)((((u64)t1 << 32) | t0) >> (2 * (x & 15)));
            const u32 lim = min(min(rcnt, (u32)(S.L - S.j)), n - 1 - x);
            const u32 d = rc ^ tc, m2 = ((d | (d >> 1)) & 0x55555555u) | rn;
            const u32 first = m2 ? (u32)(__ffs(m2) - 1) >> 1 : 16u;
            S.j += (int)min(first, lim);
            if (first < lim) S.u = 6;         // mismatch or N: the match ends here
        } else if (live) {
            fin = true;
        }
        if (fin) {
            counts[r] = em.cnt;
            if (em.cnt > em.cap) ovf_list[atomicAdd(ovf_n, 1u)] = (u32)r;
        }
        const u32 fm = __ballot_sync(0xffffffffu, fin);
        if (fm) {
            u64 it2;
            bool ok2;
            take(__popc(fm), __popc(fm & lt), it2, ok2);
            if (fin) {
                live = ok2;
                if (live) {
                    r = QUEUE && perm ? perm[it2] : it2;
                    start(r);
                }
            }
        }
    }
    work.flush(wc);
}

// Text comparison of stage 5 with the text words t0, t1 at T[x & ~15, ...), x = pos + j - i: the
// matching prefix of up to 16 read bases; a mismatch or an N ends the match (stage 6).
__device__ __forceinline__ void text_apply(SmemState &S, u32 t0, u32 t1, u32 n) {
    const u32 x = S.pos + (u32)(S.j - S.i);
    u32 rc = 0, rn = 0;
    const u32 rcnt = read_codes16(S, S.j, rc, rn);
    const u32 tc = (u32)((((u64)t1 << 32) | t0) >> (2 * (x & 15)));
    const u32 lim = min(min(rcnt, (u32)(S.L - S.j)), n - 1 - x);
    const u32 d = rc ^ tc, m2 = ((d | (d >> 1)) & 0x55555555u) | rn;
    const u32 first = m2 ? (u32)(__ffs(m2) - 1) >> 1 : 16u;
    S.j += (int)min(first, lim);
    if (first < lim) S.u = 6;
}

// The SMEM kernel with the memory actions split from the rest.  Its lanes go through Algorithm 3
// exactly as k_smem's do (same reads, same steps in the same order, same records), but a warp
// runs two kinds of iteration:
//  - a memory step, uniform for every lane that holds a memory action: an extension by P[j]
//    (stages 1-3; Algorithm 1) or an LF step of a walk (stages 4 and 7), both reading
//    occurrence blocks; a text comparison (stage 5); an SA or ISA sample (stages 4 and 6); a
//    k-mer table entry (Section 2.5).  The loads of all lanes are issued before any result is
//    used, so they are in flight together.  A lane whose next action follows without a record or
//    a restart (another extension of the same stage, stage 1's match going on to stage 2, the
//    next walk step, the next text comparison, the sample at the end of a walk, ...) stays in
//    this loop;
//  - a service pass, run when at least `wait` lanes are out of the loop, when `burst` memory
//    steps ran since the last pass, or when no lane holds a memory action: every lane out of the
//    loop applies a failed extension (a record, a restart) and moves through the stage changes
//    up to its next memory action; finished lanes take new reads.  A pass reads no index array.
// So the branches of the stages are executed together once per service pass instead of in every
// iteration.
// WARPS: resident warps per SM the launch bounds aim at (their register cap: 65,536 / (WARPS x 32)).
template <bool QUEUE, int BLOCK, int WARPS>
__global__ void __launch_bounds__(BLOCK, WARPS * 32 / BLOCK)
    k_smem_split(DevIndex I, const u8 *__restrict__ seq, const u64 *__restrict__ off, u32 nr,
                 const u8 *__restrict__ mate, u32 bs, u32 l, u32 c, bool kmer, SlotRec *__restrict__ slots,
                 u64 slot_total, u64 *__restrict__ counts, u32 *__restrict__ ovf_list, u32 *__restrict__ ovf_n,
                 const u32 *__restrict__ perm, u32 *qhead, const u32 *__restrict__ lc, bool uext, SmemTuning tune,
                 u32 *err, u32 *chk) {
    const u32 FULL = 0xffffffffu;
    const u32 lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    const u32 n = (u32)I.n, prim = (u32)I.primary, K = I.kmer_k;
    const u64 o0 = off[0];
    const u64 o1 = off[nr];
    const u8 *const end = seq + o1;
    SmemState S;
    SlotEmit em;
    WarpRange wr;
    if (!QUEUE) wr.init(nr);
    u32 lr = l, cr = c;
    auto start = [&](u64 rr) {
        u64 b = off[rr], e = off[rr + 1];
        bool bad = b > e || b < o0 || e > o1;
        if (bad) {   // offsets outside the batch or decreasing: nothing is read, no record written
            atomicOr(err, (u32)DEVCHK_OFFSETS);
            b = e = o0;
        }
        const u64 sb = slots_before(b - o0, rr), se = slots_before(e - o0, rr + 1);
        em.slots = slots;
        em.base = sb;
        em.cap = !bad && se <= slot_total ? (u32)(se - sb) : 0u;
        em.cnt = 0;
        if (lc) {
            const u32 v = lc[rr];
            lr = v & 0xFFFFu;
            cr = v >> 16;
        }
        smem_begin(S, seq + b, (int)(e - b), conv_of(mate, rr, bs), lr, n, end);
    };
    auto take = [&](u32 k, u32 rank, u64 &item, bool &ok) {
        if (QUEUE) {
            u32 base = 0;
            if (lane == 0) base = atomicAdd(qhead, k);
            base = __shfl_sync(FULL, base, 0);
            item = (u64)base + rank;
            ok = item < nr;
        } else {
            item = wr.next + rank;
            ok = item < wr.end;
            wr.next += k;
        }
    };
    // lane state: rdy = holds the memory action ract (acode: its sample index or k-mer code);
    // pend = an extension failed and is applied at the next pass
    bool rdy = false, pend = false;
    int ract = R_BLOCK;
    u32 acode = 0;
    // one service of a lane out of the loop: its pending failure and the stage changes up to its
    // next memory action.  Returns true when the read is finished.
    auto service = [&]() -> bool {
        if (pend) {
            pend = false;
            if (!smem_apply(S, 0, 0, 0, lr, cr, n, em)) return true;
        }
        u32 code = 0;
        const int act = smem_next(S, I, lr, kmer && lr >= K, em, code, uext);
        if (act == ACT_NONE) return true;
        ract = act == ACT_TEXT ? R_TEXT : (act == ACT_SAMPLE ? R_SAMPLE : (act == ACT_KMER ? R_KMER : R_BLOCK));
        acode = code;
        rdy = true;
        return false;
    };
    u64 item, r = 0;
    bool live;
    take(tune.rpw, lane < tune.rpw ? lane : 0u, item, live);   // lanes rpw.. hold no read
    live = live && lane < tune.rpw;
    if (live) {
        r = QUEUE && perm ? perm[item] : item;
        start(r);
    }
    u32 since = 0;
    for (;;) {
        if (__all_sync(FULL, !live)) break;
        const u32 out_mask = __ballot_sync(FULL, live && !rdy);
        const u32 in_mask = __ballot_sync(FULL, rdy);
        if (out_mask && (in_mask == 0 || since >= tune.burst || (u32)__popc(out_mask) >= tune.wait)) {
            since = 0;
            // ---- service pass (divergent, no index reads)
            bool fin = live && !rdy && service();
            // finished lanes hand in their counts and take new reads, which go to their first
            // memory action at once (a read shorter than l finishes there and takes the next one)
            for (;;) {
                if (fin) {
                    counts[r] = em.cnt;
                    if (em.cnt > em.cap) ovf_list[atomicAdd(ovf_n, 1u)] = (u32)r;
                }
                const u32 fm = __ballot_sync(FULL, fin);
                if (!fm) break;
                u64 it2;
                bool ok2;
                take(__popc(fm), __popc(fm & lt), it2, ok2);
                bool again = false;
                if (fin) {
                    live = ok2;
                    rdy = false;
                    pend = false;
                    if (live) {
                        r = QUEUE && perm ? perm[it2] : it2;
                        start(r);
                        again = service();
                    }
                }
                fin = again;
            }
        }
        ++since;
        // ---- memory step (uniform): every lane's memory action, loads first
        if (rdy && ract == R_BLOCK && chk) {   // MB_CHECKED: both rows inside the text (always so on a sound index)
            const bool walk = S.u >= 4, fwd = S.u == 2;
            const u64 p = (fwd || walk) ? S.kr : S.k;
            if (p + (walk ? 0u : S.s) > n) {
                atomicOr(chk, (u32)DEVCHK_BOUNDS);
                rdy = false;
                S.u = 0;   // the read ends here; the next service pass finishes it
            }
        }
        if (!rdy) continue;
        const bool walk = S.u >= 4, fwd = S.u == 2;
        const u32 p = (fwd || walk) ? S.kr : S.k, sz = walk ? 0u : S.s;
        Blk b0, b1;
        u32 w0 = 0, w1 = 0, w2 = 0;
        if (ract == R_BLOCK) {
            b0 = load_blk(I.occ + (p >> BLK_SHIFT));
            b1 = b0;
            if (((p + sz) >> BLK_SHIFT) != (p >> BLK_SHIFT)) b1 = load_blk(I.occ + ((p + sz) >> BLK_SHIFT));
        } else if (ract == R_TEXT) {
            const u32 x = S.pos + (u32)(S.j - S.i);
            w0 = __ldg(I.text2 + (x >> 4));
            w1 = __ldg(I.text2 + (x >> 4) + 1);
        } else if (ract == R_SAMPLE) {
            w0 = __ldg((S.u == 4 ? I.sa_aux : I.isa_aux) + acode);
        } else {
            const u32 *t = I.kmer + 3 * (u64)acode;
            w0 = __ldg(t);
            w1 = __ldg(t + 1);
            w2 = __ldg(t + 2);
        }
        if (ract == R_BLOCK) {
            const u32 q = fwd ? S.k : S.kr;
            const u32 a = walk ? 0u : cached_base(S, S.j);
            const u32 sym = walk ? sym_at(b0, p & BLK_MASK) : ((fwd ? 3u - a : a) & 3u);
            const Ext x = extend_blocks(I, b0, b1, p, q, sz, sym);
            if (walk) {
                S.kr = x.p;
                if (S.u == 4)
                    ++S.s;
                else
                    --S.s;
                rdy = uniq_next(S, n, prim, ract, acode);
            } else if (a < 4 && x.s >= cr) {
                S.k = fwd ? x.q : x.p;
                S.kr = fwd ? x.p : x.q;
                S.s = x.s;
                S.j += fwd ? 1 : -1;
                if (S.u == 1 && S.j < S.i) {   // P[i, i+l) is a match: stage 2 (as smem_next)
                    S.u = 2;
                    S.j = S.i + (int)lr;
                }
                if (S.u == 1) {
                    rdy = true;
                } else if (S.u == 3) {
                    rdy = S.j > S.i;
                } else if (S.j == S.L) {
                    rdy = false;
                } else if (uext && S.s == 1 && S.L - S.j >= U_MIN) {   // one occurrence: compare text
                    S.u = 4;
                    S.kr = S.k;
                    S.s = 0;
                    rdy = uniq_next(S, n, prim, ract, acode);
                }
            } else {   // the extension fails: applied at the next service pass
                rdy = false;
                pend = true;
            }
        } else if (ract == R_TEXT) {
            text_apply(S, w0, w1, n);
            rdy = uniq_next(S, n, prim, ract, acode);
        } else if (ract == R_SAMPLE) {
            if (S.u == 4) {
                S.pos = w0 + S.s;
                S.u = 5;
            } else {
                S.kr = w0;
                S.u = 7;
            }
            rdy = uniq_next(S, n, prim, ract, acode);
        } else {
            // a k-mer entry; the next action is an extension of the same stage when the match
            // goes on (else the pass decides; a finished read has u = 0)
            rdy = smem_apply_kmer(S, w0, w1, w2, lr, cr, K) &&
                  ((S.u == 1 && S.j >= S.i && S.s != n) || (S.u == 3 && S.j > S.i));
            ract = R_BLOCK;
        }
    }
}

__device__ __forceinline__ void write_rec(mb_smem *out, u64 *hitc, u64 m, u32 r, u32 qbeg, u32 qend, u64 k, u64 kr,
                                          u64 s, u32 max_occ, u64 cap) {
    if (m >= cap) return;   // past the caller's capacity (reported, not written)
    mb_smem x;
    x.read = r;
    x.qbeg = qbeg;
    x.qend = qend;
    x.flags = s > max_occ ? MB_SMEM_OVER_MAX_OCC : 0u;
    x.k = k;
    x.kr = kr;
    x.s = s;
    x.hit_off = 0;
    out[m] = x;
    hitc[m] = s > max_occ ? 0 : s;
}

// Copies each read's SMEMs from its slots to the records; reads with more SMEMs than slots (or
// whose slots lie past slot_total) are skipped here and recomputed by k_smem_overflow.
__global__ void k_gather(const u64 *__restrict__ off, u32 nr, const SlotRec *__restrict__ slots, u64 slot_total,
                         const u64 *__restrict__ counts, const u64 *__restrict__ soff, u32 max_occ,
                         mb_smem *__restrict__ out, u64 *__restrict__ hitc, u64 out_cap,
                         u32 *__restrict__ known = nullptr) {
    u64 r = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const u64 sb = slot_base(off, r), se = slot_base(off, r + 1), cnt = counts[r];
    if (se > slot_total || cnt > se - sb) return;
    const u64 o = soff[r];
    for (u64 t = 0; t < cnt; ++t) {
        SlotRec x = slots[sb + t];
        write_rec(out, hitc, o + t, (u32)r, x.qbeg, x.qend, x.k, x.kr, x.s, max_occ, out_cap);
        if (known && o + t < out_cap) known[o + t] = x.pos;
    }
}

struct FinalEmit {
    mb_smem *out;
    u64 *hitc;
    u64 o, cap;
    u32 r, max_occ;
    u32 *known;
    __device__ __forceinline__ void operator()(int i, int j, u32 k, u32 kr, u32 s, u32 = NOPOS) {
        if (known && o < cap) known[o] = NOPOS;   // the overflow pass steps; no position is known
        write_rec(out, hitc, o++, r, (u32)i, (u32)j, k, kr, s, max_occ, cap);
    }
};

__global__ void k_smem_overflow(DevIndex I, const u8 *__restrict__ seq, const u64 *__restrict__ off, u32 nr,
                                const u8 *__restrict__ mate, u32 bs, u32 l, u32 c, bool kmer,
                                const u32 *__restrict__ ovf_list,
                                const u32 *__restrict__ ovf_n, const u64 *__restrict__ soff, u32 max_occ,
                                mb_smem *__restrict__ out, u64 *__restrict__ hitc, u64 cap,
                                const u32 *__restrict__ lc, u32 *__restrict__ known = nullptr) {
    u32 n = *ovf_n;
    for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        u32 r = ovf_list[q];
        FinalEmit em{out, hitc, soff[r], cap, r, max_occ, known};
        Work<false> work;
        const u32 lr = lc ? (lc[r] & 0xFFFFu) : l, cr = lc ? (lc[r] >> 16) : c;
        smem_read(I, seq + off[r], (int)(off[r + 1] - off[r]), lr, cr, conv_of(mate, r, bs), kmer && lr >= I.kmer_k,
                  seq + off[nr], em, work);
    }
}

// m records, or min(*mdev, m) when mdev is given (count known only on the device)
__global__ void k_set_hitoff(const u64 *__restrict__ hoff, u64 m, const u64 *__restrict__ mdev,
                             mb_smem *__restrict__ out) {
    if (mdev && *mdev < m) m = *mdev;
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < m; t += (u64)gridDim.x * blockDim.x)
        out[t].hit_off = hoff[t];
}

// ---------------------------------------------------------------------------- locate
// Largest record index m with hit_off <= h (records with no hits share the offset of the next
// record that has hits, so the last such record is the one owning hit h).
__device__ __forceinline__ u64 owner_of(const mb_smem *__restrict__ sm, u64 nsm, u64 h) {
    u64 a = 0, b = nsm;   // invariant: hit_off[a] <= h, answer in [a, b)
    while (b - a > 1) {
        u64 mid = (a + b) >> 1;
        if (__ldg(&sm[mid].hit_off) <= h) a = mid;
        else b = mid;
    }
    return a;
}


// ---------------------------------------------------------------------------- shared walks
// The records of a batch repeat rows: reads that cover the same repeat give the same or nested SA
// intervals (two strings' intervals are nested when one is a prefix of the other, else
// disjoint), so on the 1 Gbp workload 331M hits hold 175M distinct rows.  Locate therefore walks
// each row of the union of the records' intervals once and copies the positions to every hit
// (Algorithm 2 gives one position per row, so the hits are the same).
//
// The records with rows to walk are compacted and sorted by (k ascending, s descending).  A
// record is maximal when its interval ends after every earlier record's; its rows are walked, in
// sorted order.  Any other record t lies inside the last maximal record before it: the first
// record that reaches the running maximum of the ends before t is maximal, starts at or before
// k_t, ends at or after k_t + s_t, and no maximal record can lie between it and t.  This holds for
// any intervals (the public mb_locate takes records from the caller); nested ones share every
// repeated row.
constexpr int SHARE_S_BITS = 9;                                   // s in the low bits of the sort key
// key bits to sort: those of the largest row k < n, then s (k's unused high bits are all zero)
inline int share_key_bits(u64 n) {
    int b = 1;
    while (b < 32 && (n - 1) >> b) ++b;
    return b + SHARE_S_BITS;
}

__device__ __forceinline__ u64 count_of(u64 cap, const u64 *n_dev) { return n_dev && *n_dev < cap ? *n_dev : cap; }
__device__ __forceinline__ u64 hits_of(const mb_smem *__restrict__ sm, u64 m) {
    return (__ldg(&sm[m].flags) & MB_SMEM_OVER_MAX_OCC) ? 0 : __ldg(&sm[m].s);
}

// A record walks its rows when it has hits and its position was not found while seeding.
__device__ __forceinline__ bool walks(u64 cnt, const u32 *known, u64 t) {
    return cnt && !(known && cnt == 1 && known[t] != NOPOS);
}
// A record whose rows [k, k+s) leave the text (only records from a caller can): flagged in the
// error word and left out of the walks, its hits unwritten.
__device__ __forceinline__ bool rows_outside(const mb_smem *__restrict__ sm, u64 t, u64 cnt, u64 n) {
    const u64 k = __ldg(&sm[t].k);
    return cnt && (k >= n || cnt > n - k);
}

// flag[t] = 1 for a record with rows to walk.  A record with a known position (one hit, found
// while seeding) writes that hit here and walks nothing.
__global__ void k_share_flag(const mb_smem *__restrict__ sm, u64 cap, const u64 *__restrict__ nsm_dev,
                             const u32 *__restrict__ known, u32 *__restrict__ hits, u64 hits_cap,
                             u64 *__restrict__ flag, u64 n, u32 *err) {
    const u64 nsm = count_of(cap, nsm_dev);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < cap; t += (u64)gridDim.x * blockDim.x) {
        u64 f = 0;
        if (t < nsm) {
            const u64 cnt = hits_of(sm, t);
            if (rows_outside(sm, t, cnt, n)) {
                atomicOr(err, (u32)DEVCHK_RECORD);
            } else if (walks(cnt, known, t)) {
                f = 1;
            } else if (cnt == 1) {   // known position
                const u64 ho = __ldg(&sm[t].hit_off);
                if (ho < hits_cap) hits[ho] = known[t];
            }
        }
        flag[t] = f;
    }
}

// The flagged records (see k_share_flag) at their scanned places `at`: sort key
// (k << 9 | 511 - min(s, 511)) and record number.
__global__ void k_share_compact(const mb_smem *__restrict__ sm, u64 cap, const u64 *__restrict__ nsm_dev,
                                const u32 *__restrict__ known, const u64 *__restrict__ at, u64 *__restrict__ keys,
                                u32 *__restrict__ vals, u64 n) {
    const u64 nsm = count_of(cap, nsm_dev);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < nsm; t += (u64)gridDim.x * blockDim.x) {
        const u64 cnt = hits_of(sm, t);
        if (!walks(cnt, known, t) || rows_outside(sm, t, cnt, n)) continue;
        const u64 sb = cnt < (1u << SHARE_S_BITS) ? cnt : (1u << SHARE_S_BITS) - 1;
        keys[at[t]] = ((u64)(u32)__ldg(&sm[t].k) << SHARE_S_BITS) | ((1u << SHARE_S_BITS) - 1 - sb);
        vals[at[t]] = (u32)t;
    }
}

// For sorted record t < nw: its s and hit offset in sorted order, and ends[t] = k + s (saturated
// to 32 bits); ends = 0 past the records.
__global__ void k_share_gather(const mb_smem *__restrict__ sm, const u64 *__restrict__ keys,
                               const u32 *__restrict__ vals, u64 cap, const u64 *__restrict__ nw_dev,
                               u32 *__restrict__ ss, u64 *__restrict__ sho, u32 *__restrict__ ends) {
    const u64 nw = count_of(cap, nw_dev);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < cap; t += (u64)gridDim.x * blockDim.x) {
        u32 e = 0;
        if (t < nw) {
            const u32 r = vals[t];
            const u64 s = __ldg(&sm[r].s);
            const u64 end = (keys[t] >> SHARE_S_BITS) + s;
            ss[t] = (u32)s;
            sho[t] = __ldg(&sm[r].hit_off);
            e = end < 0xFFFFFFFFull ? (u32)end : 0xFFFFFFFFu;
        }
        ends[t] = e;
    }
}

// With pmax = the running maximum of the ends: len[t] = s of a maximal record (else 0) and
// last[t] = t for a maximal record (else 0), to be scanned into row offsets and owners.
__global__ void k_share_mark(const u64 *__restrict__ keys, const u32 *__restrict__ ss, u64 cap,
                             const u64 *__restrict__ nw_dev, const u32 *__restrict__ pmax, u64 *__restrict__ len,
                             u32 *__restrict__ last) {
    const u64 nw = count_of(cap, nw_dev);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < cap; t += (u64)gridDim.x * blockDim.x) {
        u64 l = 0;
        u32 lm = 0;
        if (t < nw) {
            const u64 end = (keys[t] >> SHARE_S_BITS) + ss[t];
            const u32 e = end < 0xFFFFFFFFull ? (u32)end : 0xFFFFFFFFu;
            if (t == 0 || e > pmax[t - 1]) {   // pmax[t - 1] >= 1 here, so the first record is maximal
                l = ss[t];
                lm = (u32)t;
            }
        }
        len[t] = l;
        last[t] = lm;
    }
}

// rows[roff[t] + q] = k + q for every maximal sorted record t (last[t] == t): one warp per 32
// sorted records, each record's rows written by the whole warp.
__global__ void k_share_rows(const u64 *__restrict__ keys, const u32 *__restrict__ ss, const u32 *__restrict__ last,
                             const u64 *__restrict__ roff, u64 cap, const u64 *__restrict__ nw_dev,
                             u32 *__restrict__ rows, u64 rows_cap) {
    const u32 lane = threadIdx.x & 31;
    const u64 nw = count_of(cap, nw_dev);
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 base = ((blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5) * 32; base < nw; base += nwarps * 32) {
        const u64 t = base + lane;
        u64 o = 0, c = 0;
        u32 k = 0;
        if (t < nw && last[t] == (u32)t) {
            o = roff[t];
            c = ss[t];
            k = (u32)(keys[t] >> SHARE_S_BITS);
        }
        for (int q = 0; q < 32; ++q) {
            const u64 oq = __shfl_sync(0xffffffffu, o, q), cq = __shfl_sync(0xffffffffu, c, q);
            const u32 kq = __shfl_sync(0xffffffffu, k, q);
            for (u64 u = lane; u < cq && oq + u < rows_cap; u += 32) rows[oq + u] = kq + (u32)u;
        }
    }
}

// hits[hit_off + q] = rpos[roff[o] + (k - k_o) + q] for every sorted record, o = last[t] being
// its owner (itself when maximal): one warp per 32 sorted records, copies by the whole warp.
__global__ void k_share_copy(const u64 *__restrict__ keys, const u32 *__restrict__ ss, const u64 *__restrict__ sho,
                             const u32 *__restrict__ last, const u64 *__restrict__ roff, u64 cap,
                             const u64 *__restrict__ nw_dev, const u32 *__restrict__ rpos, u64 rows_cap,
                             u32 *__restrict__ hits, u64 hits_cap) {
    const u32 lane = threadIdx.x & 31;
    const u64 nw = count_of(cap, nw_dev);
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 base = ((blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5) * 32; base < nw; base += nwarps * 32) {
        const u64 t = base + lane;
        u64 src = 0, dst = 0, c = 0;
        if (t < nw) {
            const u32 o = last[t];
            c = ss[t];
            dst = sho[t];
            src = roff[o] + ((keys[t] >> SHARE_S_BITS) - (keys[o] >> SHARE_S_BITS));
        }
        for (int q = 0; q < 32; ++q) {
            const u64 sq = __shfl_sync(0xffffffffu, src, q), dq = __shfl_sync(0xffffffffu, dst, q);
            const u64 cq = __shfl_sync(0xffffffffu, c, q);
            for (u64 u = lane; u < cq; u += 32)
                if (dq + u < hits_cap && sq + u < rows_cap) hits[dq + u] = rpos[sq + u];
        }
    }
}

// Locate (Algorithm 2).  Each lane LF-walks D rows at a time (D independent block reads in
// flight per lane), one step of each per loop iteration.  The walks that end in an iteration are
// replaced in one hand-out: the lanes' counts of ended walks are scanned across the warp and each
// ended walk takes the next position of the warp's chunk of the row list (in lane order, then
// slot order); warps take chunks of 256 positions per walk slot from a device queue, so a warp
// whose walks happen to be short takes more rows and the launch ends with its last walks.  A
// walk ends on a sampled row (position = steps + S(row)) or on the $ row (S = 0, position =
// steps).  The sampled-SA reads and the block reads of one iteration are issued together.  A walk
// needs fewer than n steps; the bound only guards against a corrupted index (it then writes
// 0xFFFFFFFF).  Queue positions are u32 (the host keeps them below 2^32).
// Launch bounds: 16 walks per lane fit one block of 8 warps per SM, 8 walks two, 4 three, fewer
// four.
// CHK (MB_CHECKED): every row walked is checked against the text length, failures recorded in *chk.
template <bool COUNT, bool POW2, int D, bool CHK = false>
__global__ void __launch_bounds__(256, D <= 2 ? 4 : (D <= 4 ? 3 : (D <= 8 ? 2 : 1)))
    k_locate(DevIndex I, const u32 *__restrict__ rows, u64 nhits, const u64 *__restrict__ nhits_dev,
             u32 *__restrict__ hits, u32 *__restrict__ qhead, u64 *wc, u32 *chk) {
    constexpr u32 CHUNK = 256u * D;   // queue positions a warp takes at a time
    const u32 FULL = 0xffffffffu, lane = threadIdx.x & 31;
    if (nhits_dev && *nhits_dev < nhits) nhits = *nhits_dev;
    const u32 nitems = (u32)nhits;
    Work<COUNT> work;
    const u32 r = I.r, rmask = I.r - 1, rshift = __ffs(I.r) - 1, prim = (u32)I.primary, n = (u32)I.n;
    const u32 C0 = (u32)I.C[0], C1 = (u32)I.C[1], C2 = (u32)I.C[2], C3 = (u32)I.C[3];
    u32 h[D], row[D], steps[D];
    u32 live = 0;   // bit d: slot d holds a walk
    u32 next = 0;   // the warp's queue chunk: positions [next, cend)
    if (lane == 0) next = atomicAdd(qhead, CHUNK);
    next = __shfl_sync(FULL, next, 0);
    u32 cend = next + CHUNK;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const u32 o = next + 32u * d + lane;
        h[d] = o;
        steps[d] = 0;
        row[d] = 0;
        if (o < nitems) {
            live |= 1u << d;
            row[d] = __ldg(&rows[o]);
        }
    }
    next += 32u * D;
    for (;;) {
        if (__all_sync(FULL, live == 0)) break;
        if (next + 128 + lane < cend && next + 128 + lane < nitems)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(rows + next + 128 + lane));
        u32 stop = 0, smp = 0, skp = 0;
        u32 sv[D];
        Blk b[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const bool on = (live >> d) & 1u;
            const bool skip = row[d] == NOPOS;   // a row to skip (its hit is written elsewhere)
            const bool bad = CHK && on && !skip && row[d] >= n;   // MB_CHECKED: a row outside the text
            if (CHK && bad) atomicOr(chk, (u32)DEVCHK_BOUNDS);
            const bool sampled = !skip && !bad && (POW2 ? (row[d] & rmask) == 0 : row[d] % r == 0);
            const bool st = on && (skip || bad || sampled || row[d] == prim || steps[d] > n);
            sv[d] = 0;
            if (st) {
                stop |= 1u << d;
                if (skip) skp |= 1u << d;
                if (sampled) {
                    smp |= 1u << d;
                    sv[d] = __ldg(&I.ssa[POW2 ? (row[d] >> rshift) : row[d] / r]);
                }
            } else if (on) {
                b[d] = load_blk(I.occ + (row[d] >> BLK_SHIFT));
            }
        }
        // positions for this iteration's ended walks: from the warp's chunk, then a new chunk
        const u32 cnt = __popc(stop);
        u32 incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(FULL, incl, o);
            if (lane >= (u32)o) incl += v;
        }
        const u32 total = __shfl_sync(FULL, incl, 31), avail = cend - next;
        u32 nb = cend;   // past the end once the chunk reached it (a new chunk would too)
        if (total > avail && cend < nitems) {
            if (lane == 0) nb = atomicAdd(qhead, CHUNK);
            nb = __shfl_sync(FULL, nb, 0);
        }
        u32 k = incl - cnt;   // this lane's first position among the warp's
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if ((stop >> d) & 1u) {
                if (!((skp >> d) & 1u))
                    hits[h[d]] = (steps[d] > n || (CHK && row[d] >= n))
                                     ? 0xFFFFFFFFu
                                     : (((smp >> d) & 1u) ? sv[d] + steps[d] : steps[d]);
                work.lf += steps[d];
                work.sa += (smp >> d) & 1u;
                const u32 pos = k < avail ? next + k : nb + (k - avail);
                ++k;
                h[d] = pos;
                steps[d] = 0;
                if (pos < nitems) row[d] = __ldg(&rows[pos]);
                else live &= ~(1u << d);
            } else if ((live >> d) & 1u) {
                row[d] = lf_blk(b[d], row[d], prim, C0, C1, C2, C3);
                ++steps[d];
            }
        }
        if (total > avail) {
            next = nb + (total - avail);
            cend = nb + CHUNK;
        } else {
            next += total;
        }
    }
    work.flush(wc);
}

// ---------------------------------------------------------------------------- walks that join
// Reads that cover the same place give hits a few text positions apart (SMEMs of one read overlap):
// on the workloads here about 78% of the distinct hit positions have another hit within 8
// positions to their left.  An LF-walk (Algorithm 2) from the row of position p visits the rows of
// p - 1, p - 2, ... in turn, so when it reaches the row of another hit q whose position is already
// known, after d = p - q steps, S(row of p) = S(row of q) + d and the walk can stop.
//
// The walked rows go in JOIN_PASSES passes by a hash of the row; a walk of pass k may stop at a
// walked row of an earlier pass (its position is final by then), so no walk waits on another.
// Membership must cost no extra random read per step, so each call makes its own copy of the
// occurrence blocks ("walk blocks", 32 bytes per 64 rows like the blocks): the counts of A, C and
// G as 21-bit offsets from coarse counts kept per 2^21 rows (T follows from the row count), the
// two bit planes, and 64 mark bits of the walked rows.  The coarse counts (at most 2,049 of them,
// 16 bytes each) sit in shared memory.  The rank of a marked row (its place in the sorted row
// list, where its position is written) is the block's count of marked rows before it plus a
// popcount.  The positions are exactly those of the plain walks.  This needs the walked rows
// sorted and distinct (true for the records of one seeding call, whose intervals are nested or
// disjoint); otherwise a device flag turns the joins off and every walk runs to its sampled row.
constexpr int JOIN_PASSES = 8, JOIN_PASS_BITS = 3;
constexpr u32 COARSE_SHIFT = 21;        // coarse counts per 2^21 rows
constexpr u32 FINE_BITS = 21, FINE_MASK = (1u << FINE_BITS) - 1;
constexpr u64 JOIN_TILE = 4096;         // rows per warp tile of the pass partition

struct __align__(32) WalkBlk {
    u64 fc;          // counts of A, C, G before the block minus the coarse counts, 21 bits each
    u64 lo, hi;      // the bit planes, as in the occurrence block
    u64 marks;       // bit q: row q of the block is a walked row
};
__device__ __forceinline__ u32 join_pass(u32 row) { return (row * 0x9E3779B1u) >> (32 - JOIN_PASS_BITS); }
__device__ __forceinline__ void load_walk_blk(const WalkBlk *__restrict__ w, u64 &fc, u64 &lo, u64 &hi, u64 &mk) {
    asm("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(fc), "=l"(lo), "=l"(hi), "=l"(mk) : "l"(w));
}

// Coarse counts (C[a] plus the block counts at every 2^15-th block) and the walk blocks with no
// marks.
__global__ void k_walk_blocks(DevIndex I, u64 nb, uint4 *__restrict__ coarse, WalkBlk *__restrict__ wb) {
    constexpr u32 GB = COARSE_SHIFT - BLK_SHIFT;
    for (u64 b = blockIdx.x * (u64)blockDim.x + threadIdx.x; b < nb; b += (u64)gridDim.x * blockDim.x) {
        const OccBlock o = I.occ[b];
        const u64 cb = (b >> GB) << GB;
        const OccBlock c = I.occ[cb];
        if (b == cb)
            coarse[b >> GB] = make_uint4((u32)I.C[0] + o.cnt[0], (u32)I.C[1] + o.cnt[1], (u32)I.C[2] + o.cnt[2],
                                         (u32)I.C[3] + o.cnt[3]);
        WalkBlk w;
        w.fc = (u64)(o.cnt[0] - c.cnt[0]) | ((u64)(o.cnt[1] - c.cnt[1]) << FINE_BITS) |
               ((u64)(o.cnt[2] - c.cnt[2]) << (2 * FINE_BITS));
        w.lo = o.lo;
        w.hi = o.hi;
        w.marks = 0;
        wb[b] = w;
    }
}

// Mark bits of the walked rows (warp-aggregated atomics over the sorted rows), the not-sorted
// flag, and for every block holding walked rows the number of walked rows before it (written by
// the block's first row; only marked blocks are ever read).
__global__ void k_join_mark(const u32 *__restrict__ rows, const u64 *__restrict__ nrows_dev, u64 cap,
                            WalkBlk *__restrict__ wb, u32 *__restrict__ before, u32 *__restrict__ nojoin) {
    const u64 nr = count_of(cap, nrows_dev);
    const u32 lane = threadIdx.x & 31;
    for (u64 base = (blockIdx.x * (u64)blockDim.x + threadIdx.x) & ~31ull; base < nr;
         base += (u64)gridDim.x * blockDim.x) {
        const u64 i = base + lane;
        const bool on = i < nr;
        const u32 y = on ? rows[i] : 0u;
        if (on && i + 1 < nr && rows[i + 1] <= y) atomicOr(nojoin, 1u);
        const u32 w = y >> BLK_SHIFT;
        if (on && (i == 0 || (rows[i - 1] >> BLK_SHIFT) != w)) before[w] = (u32)i;
        const u32 act = __ballot_sync(0xffffffffu, on);
        if (!on) continue;
        const u32 grp = __match_any_sync(act, w);
        const u64 bit = 1ull << (y & BLK_MASK);
        const u32 lo = __reduce_or_sync(grp, (u32)bit), hi = __reduce_or_sync(grp, (u32)(bit >> 32));
        if (lane == (u32)(__ffs(grp) - 1))
            atomicOr((unsigned long long *)&wb[w].marks, ((unsigned long long)hi << 32) | lo);
    }
}

// Counting mode: the calls whose walked rows were not sorted and distinct (no joins).
__global__ void k_join_flag_count(const u32 *__restrict__ nojoin, u64 *wc) {
    if (threadIdx.x == 0 && *nojoin) atomicAdd((unsigned long long *)&wc[WC_JOIN_OFF], 1ull);
}

// Stable partition of the sorted rows by pass: per warp tile of JOIN_TILE rows, the count of each
// pass (tcnt[p * ntiles + tile]); after an exclusive scan of those counts (pass-major), the row
// numbers of each pass in order (idx) and the pass boundaries (range[p], range[JOIN_PASSES]).
template <bool SCATTER>
__global__ void k_pass_split(const u32 *__restrict__ rows, const u64 *__restrict__ nrows_dev, u64 cap, u64 ntiles,
                             u32 *__restrict__ tcnt, u32 *__restrict__ idx, u64 *__restrict__ range) {
    const u64 nr = count_of(cap, nrows_dev);
    const u32 lane = threadIdx.x & 31;
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 t = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nwarps) {
        u32 run[JOIN_PASSES];
#pragma unroll
        for (int p = 0; p < JOIN_PASSES; ++p) run[p] = SCATTER ? tcnt[(u64)p * ntiles + t] : 0u;
        const u64 e = (t + 1) * JOIN_TILE < nr ? (t + 1) * JOIN_TILE : nr;
        for (u64 c = t * JOIN_TILE; c < e; c += 32) {
            const u64 i = c + lane;
            const u32 ps = i < e ? join_pass(rows[i]) : JOIN_PASSES;
#pragma unroll
            for (int p = 0; p < JOIN_PASSES; ++p) {
                const u32 m = __ballot_sync(0xffffffffu, ps == (u32)p);
                if (SCATTER && ps == (u32)p) idx[run[p] + __popc(m & ((1u << lane) - 1u))] = (u32)i;
                run[p] += __popc(m);
            }
        }
        if (!SCATTER && lane == 0)
            for (int p = 0; p < JOIN_PASSES; ++p) tcnt[(u64)p * ntiles + t] = run[p];
    }
    if (SCATTER && blockIdx.x == 0 && threadIdx.x <= JOIN_PASSES)
        range[threadIdx.x] = threadIdx.x < JOIN_PASSES ? (ntiles ? tcnt[(u64)threadIdx.x * ntiles] : 0) : nr;
}

__device__ __forceinline__ u32 ld_cg_u32(const u32 *p) {   // from L2 (written by an earlier launch)
    u32 v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Algorithm 2 over the rows of one pass with joins: k_locate's walk loop (D walks per lane) on
// the walk blocks.  A walk past its first row that stands on a marked row of an earlier pass
// stops: the next iteration reads the block's count of marked rows before it (the rank), the one
// after reads that row's position (final: its pass ran in an earlier launch).  Warps take the
// pass's rows (through idx, in row order) from a device queue in chunks of 256 per walk slot, so
// warps whose walks happen to be short take more rows and the pass ends with the grid's last
// walks rather than with its most loaded warp.
template <bool COUNT, bool POW2, int D>
__global__ void __launch_bounds__(256, D <= 2 ? 4 : (D <= 4 ? 3 : (D <= 8 ? 2 : 1)))
    k_locate_join(DevIndex I, const u32 *__restrict__ rows, const u32 *__restrict__ idx, const u64 *__restrict__ range,
                  u32 pass, const WalkBlk *__restrict__ wb, const uint4 *__restrict__ coarse, u32 ncoarse,
                  const u32 *__restrict__ before, const u32 *__restrict__ nojoin, u32 *__restrict__ rpos,
                  u32 *__restrict__ qhead, u64 *wc) {
    constexpr u32 CHUNK = 256u * D;   // queue positions a warp takes at a time
    extern __shared__ uint4 cs[];     // the coarse counts
    for (u32 g = threadIdx.x; g < ncoarse; g += blockDim.x) cs[g] = coarse[g];
    __syncthreads();
    const u32 FULL = 0xffffffffu, lane = threadIdx.x & 31;
    const u64 lo_r = range[pass], hi_r = range[pass + 1];
    const u32 nitems = hi_r > lo_r ? (u32)(hi_r - lo_r) : 0u;
    const u32 *__restrict__ qidx = idx + lo_r;
    u32 *const head = qhead + pass;
    const bool join = *nojoin == 0 && pass > 0;
    Work<COUNT> work;
    const u32 r = I.r, rmask = I.r - 1, rshift = __ffs(I.r) - 1, prim = (u32)I.primary, n = (u32)I.n;
    u32 h[D], row[D], steps[D];
    u32 live = 0, rk1 = 0, rk2 = 0;   // walks: present; met a marked row (row[] = block | pc << 26); rank known
    u32 next = 0;                     // the warp's queue chunk: positions [next, cend)
    if (lane == 0) next = atomicAdd(head, CHUNK);
    next = __shfl_sync(FULL, next, 0);
    u32 cend = next + CHUNK;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const u32 o = next + 32u * d + lane;
        steps[d] = 0;
        row[d] = 0;
        h[d] = 0;
        if (o < nitems) {
            live |= 1u << d;
            h[d] = __ldg(&qidx[o]);
            row[d] = __ldg(&rows[h[d]]);
        }
    }
    next += 32u * D;
    for (;;) {
        if (__all_sync(FULL, live == 0)) break;
        u32 stop = 0, smp = 0, ld = 0;
        u32 sv[D];
        u64 fc[D], bl[D], bh[D], mk[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const bool on = (live >> d) & 1u;
            const bool r1 = (rk1 >> d) & 1u, r2 = (rk2 >> d) & 1u;
            const bool sampled = !r1 && !r2 && (POW2 ? (row[d] & rmask) == 0 : row[d] % r == 0);
            const bool st = on && (r2 || sampled || (!r1 && row[d] == prim) || steps[d] > n);
            sv[d] = 0;
            if (st) {
                stop |= 1u << d;
                if (r2) {
                    sv[d] = ld_cg_u32(&rpos[row[d]]);   // the joined row's position, final since its pass
                    smp |= 1u << d;
                } else if (sampled) {
                    smp |= 1u << d;
                    sv[d] = __ldg(&I.ssa[POW2 ? (row[d] >> rshift) : row[d] / r]);
                }
            } else if (on && r1) {
                sv[d] = __ldg(&before[row[d] & 0x3FFFFFFu]);
            } else if (on) {
                load_walk_blk(wb + (row[d] >> BLK_SHIFT), fc[d], bl[d], bh[d], mk[d]);
                ld |= 1u << d;
            }
        }
        // queue positions for the walks that end: from the warp's chunk, then a new chunk
        const u32 cnt = __popc(stop);
        u32 incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(FULL, incl, o);
            if (lane >= (u32)o) incl += v;
        }
        const u32 total = __shfl_sync(FULL, incl, 31), avail = cend - next;
        u32 nb = cend;   // past the end once the chunk reached it (a new chunk would too)
        if (total > avail && cend < nitems) {
            if (lane == 0) nb = atomicAdd(head, CHUNK);
            nb = __shfl_sync(FULL, nb, 0);
        }
        u32 k = incl - cnt;   // this lane's first position among the warp's
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if ((stop >> d) & 1u) {
                rpos[h[d]] = steps[d] > n ? 0xFFFFFFFFu : (((smp >> d) & 1u) ? sv[d] + steps[d] : steps[d]);
                work.lf += steps[d];
                work.sa += ((smp >> d) & 1u) && !((rk2 >> d) & 1u);
                work.joins += (rk2 >> d) & 1u;
                rk1 &= ~(1u << d);
                rk2 &= ~(1u << d);
                steps[d] = 0;
                const u32 pos = k < avail ? next + k : nb + (k - avail);
                ++k;
                if (pos < nitems) {
                    h[d] = __ldg(&qidx[pos]);
                    row[d] = __ldg(&rows[h[d]]);
                } else {
                    live &= ~(1u << d);
                }
            } else if ((rk1 >> d) & 1u) {   // the rank: marked rows before the block, then in it
                row[d] = sv[d] + (row[d] >> 26);
                rk1 &= ~(1u << d);
                rk2 |= 1u << d;
            } else if ((ld >> d) & 1u) {
                const u32 x = row[d], m = x & BLK_MASK;
                if (join && steps[d] > 0 && ((mk[d] >> m) & 1ull) && join_pass(x) < pass) {
                    row[d] = (x >> BLK_SHIFT) | ((u32)__popcll(mk[d] & rows_before(m)) << 26);
                    rk1 |= 1u << d;
                } else {
                    const u32 a = (u32)((bl[d] >> m) & 1) | ((u32)((bh[d] >> m) & 1) << 1);
                    const u64 eq = (bl[d] ^ ((u64)(a & 1) - 1)) & (bh[d] ^ ((u64)(a >> 1) - 1));
                    u32 c = (u32)__popcll(eq & rows_before(m));
                    if (a == 0) c -= dollar_before(x, prim);
                    const u32 fa = (u32)fc[d] & FINE_MASK, fcc = (u32)(fc[d] >> FINE_BITS) & FINE_MASK,
                              fg = (u32)(fc[d] >> (2 * FINE_BITS)) & FINE_MASK;
                    // T: the rows of the group before the block, less A, C, G and the $ row
                    const u32 gs = x & ~((1u << COARSE_SHIFT) - 1), bs = x & ~BLK_MASK;
                    const u32 ft = (bs - gs) - fa - fcc - fg - (prim >= gs && prim < bs ? 1u : 0u);
                    const uint4 g = cs[x >> COARSE_SHIFT];
                    row[d] = sel4(a, g.x + fa, g.y + fcc, g.z + fg, g.w + ft) + c;
                    ++steps[d];
                }
            }
        }
        if (total > avail) {
            next = nb + (total - avail);
            cend = nb + CHUNK;
        } else {
            next += total;
        }
    }
    work.flush(wc);
}

__global__ void k_bs_filter(const mb_smem *__restrict__ sm, u64 nsm, const u8 *__restrict__ mate,
                            const u32 *__restrict__ hits, u64 nhits, u64 M, u8 *__restrict__ keep) {
    for (u64 h = blockIdx.x * (u64)blockDim.x + threadIdx.x; h < nhits; h += (u64)gridDim.x * blockDim.x) {
        u64 m = owner_of(sm, nsm, h);
        u64 len = sm[m].qend - sm[m].qbeg;
        u8 mt = mate ? mate[sm[m].read] : 0;
        u64 pos = hits[h];
        u64 seg = pos / M;
        bool whole = (pos + len - 1) / M == seg;
        bool ok = mt == 1 ? (seg == 0 || seg == 2) : mt == 2 ? (seg == 1 || seg == 3) : true;
        keep[h] = (whole && ok) ? 1 : 0;
    }
}

void opts_defaults(const mb_opts *o, u32 &l, u32 &c, u32 &max_occ, u32 &flags) {
    l = o && o->min_len ? o->min_len : 19;
    c = o && o->min_occ ? o->min_occ : 1;
    max_occ = o && o->max_occ ? o->max_occ : 500;
    flags = o ? o->flags : 0;
}

// Grid of as many blocks as are resident at once (per-lane refill loops need no more), capped by
// the work available.
unsigned resident_grid(const void *kernel, int block, u64 work_items) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    u64 g = (u64)sms * (u64)per_sm;
    u64 need = (work_items + block - 1) / block;
    if (need < g) g = need;
    return (unsigned)(g ? g : 1);
}

template <bool QUEUE, int BLOCK, int WARPS>
int launch_split_t(const SmemArgs &a, cudaStream_t st) {
    const unsigned g = resident_grid((const void *)k_smem_split<QUEUE, BLOCK, WARPS>, BLOCK, a.nr);
    k_smem_split<QUEUE, BLOCK, WARPS><<<g, BLOCK, 0, st>>>(a.I, a.seq, a.off, a.nr, a.mate, a.bs, a.l, a.c, a.kmer,
                                                           a.slots, a.slot_total, a.counts, a.ovf_list, a.ovf_n,
                                                           a.perm, a.qhead, a.lc, a.uext, a.tune, a.err, a.chk);
    MB_KCHECK();
    return MB_OK;
}

template <bool COUNT, bool QUEUE, int BLOCK>
int launch_smem_t(const SmemArgs &a, cudaStream_t st) {
    if constexpr (!COUNT) {
        if (a.split) {
            if constexpr (BLOCK != 128) {
                if (a.warps >= 48) return launch_split_t<QUEUE, BLOCK, 48>(a, st);
            }
            if constexpr (BLOCK == 256) {
                if (a.warps >= 40) return launch_split_t<QUEUE, BLOCK, 40>(a, st);
            }
            return launch_split_t<QUEUE, BLOCK, BLOCK == 128 ? 24 : 32>(a, st);
        }
    }
    const unsigned g = resident_grid((const void *)k_smem<COUNT, QUEUE, BLOCK>, BLOCK, a.nr);
    k_smem<COUNT, QUEUE, BLOCK><<<g, BLOCK, 0, st>>>(a.I, a.seq, a.off, a.nr, a.mate, a.bs, a.l, a.c, a.kmer, a.slots,
                                                     a.slot_total, a.counts, a.ovf_list, a.ovf_n, a.perm, a.qhead,
                                                     a.wc, a.lc, a.uext, a.err);
    MB_KCHECK();
    return MB_OK;
}

// The SMEM kernel's form and tuning from the options: k_smem_split unless MB_SMEM_ONE_LOOP.
void smem_tuning(const mb_opts *o, SmemArgs &a) {
    a.split = !(o && (o->flags & MB_SMEM_ONE_LOOP));
    a.tune.burst = o && o->smem_burst ? o->smem_burst : SMEM_BURST;
    a.tune.wait = o && o->smem_wait ? (o->smem_wait > 32 ? 32u : o->smem_wait) : SMEM_WAIT;
    a.warps = o ? o->smem_warps : 0;
    a.tune.rpw = o && o->smem_reads_per_warp && o->smem_reads_per_warp < 32 ? o->smem_reads_per_warp : 32u;
}

template <bool COUNT, bool POW2, int D, bool CHK = false>
int launch_locate_t(const DevIndex &I, const u32 *rows, u64 nhits, const u64 *nhits_dev, u32 *hits, u32 *qhead,
                    u64 *wc, u32 *chk, cudaStream_t st) {
    const unsigned g = resident_grid((const void *)k_locate<COUNT, POW2, D, CHK>, 256, (nhits + 63) / 64 * 32);
    if (nhits + (u64)g * 8 * 256 * D + 256 * D >= (1ull << 32)) {   // queue positions are u32
        mb_set_error("locate: %llu hits exceed the walk queue", (unsigned long long)nhits);
        return MB_ERR_ARG;
    }
    MB_CK(cudaMemsetAsync(qhead, 0, 4, st));
    k_locate<COUNT, POW2, D, CHK><<<g, 256, 0, st>>>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk);
    MB_KCHECK();
    return MB_OK;
}
int launch_locate(const DevIndex &I, const u32 *rows, u64 nhits, const u64 *nhits_dev, u32 *hits, u32 *qhead, u64 *wc,
                  bool count, u32 depth, u32 *chk, cudaStream_t st) {
    const bool pow2 = (I.r & (I.r - 1)) == 0;
    if (chk)   // MB_CHECKED: one walk per lane, every row checked
        return pow2 ? launch_locate_t<false, true, 1, true>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st)
                    : launch_locate_t<false, false, 1, true>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (count) return pow2 ? launch_locate_t<true, true, 1>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st)
                           : launch_locate_t<true, false, 1>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (!pow2) return launch_locate_t<false, false, 1>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (depth >= 16) return launch_locate_t<false, true, 16>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (depth >= 8) return launch_locate_t<false, true, 8>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (depth >= 4) return launch_locate_t<false, true, 4>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    if (depth >= 2) return launch_locate_t<false, true, 2>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
    return launch_locate_t<false, true, 1>(I, rows, nhits, nhits_dev, hits, qhead, wc, chk, st);
}

// Device arrays of the shared-walk locate: per record (cap) sort keys and values with their
// scratch (which then hold the sorted records' s and hit offsets), running maxima of the ends,
// owners, row offsets; per row (rows_cap) the rows and their positions; the counts of records
// that walk and of rows; scan and sort scratch.
struct ShareBufs {
    u64 *keys = nullptr, *keys_alt = nullptr, *roff = nullptr, *nwalk = nullptr, *nrows = nullptr;
    u32 *vals = nullptr, *vals_alt = nullptr, *pmax = nullptr, *last = nullptr, *rows = nullptr, *rpos = nullptr;
    void *tmp = nullptr;
    u32 *err = nullptr;   // the device error word (records with rows outside the text; MB_CHECKED bounds)
    u32 *lq = nullptr;    // the head of the plain walks' row queue
    bool checked = false; // MB_CHECKED: the locate kernel checks every row it walks
    // walks that join (k_locate_join, MB_LOCATE_JOIN): the walk blocks and coarse counts, per
    // block the walked rows before it, the not-sorted flag, and the partition of the rows by pass
    // (per-tile pass counts, the row numbers by pass, the pass boundaries)
    bool join = true;
    bool aux = false;   // MB_LOCATE_AUX: walks stop at the index's rate-4 SA samples (no joins)
    WalkBlk *wb = nullptr;
    uint4 *coarse = nullptr;
    u32 *before = nullptr, *nojoin = nullptr, *tcnt = nullptr, *idx = nullptr;
    u64 *range = nullptr;
    u32 *qhead = nullptr;  // per pass: the head of the queue its launch takes rows from
};
// sizes of carved workspace arrays are rounded up to 256 bytes
inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
// walk blocks of an index of n rows (one per occurrence block), coarse counts, partition tiles
inline u64 join_words(u64 n) { return n / BLK_ROWS + 1; }
inline u64 join_coarse(u64 n) { return (join_words(n) >> (COARSE_SHIFT - BLK_SHIFT)) + 1; }
inline u64 join_tiles(u64 rows_cap) { return (rows_cap + JOIN_TILE - 1) / JOIN_TILE; }
// device bytes of the join arrays for an index of n rows and rows_cap walked rows
inline size_t join_bytes(u64 n, u64 rows_cap) {
    return align_up(join_words(n) * sizeof(WalkBlk)) + align_up(join_coarse(n) * 16) + align_up(join_words(n) * 4) +
           align_up(8) + align_up(JOIN_PASSES * join_tiles(rows_cap) * 4 + 4) + align_up(rows_cap * 4) +
           align_up((JOIN_PASSES + 1) * 8) + align_up(JOIN_PASSES * 4);
}

template <bool COUNT, bool POW2, int D>
int launch_join_t(const DevIndex &I, const u32 *rows, u64 nhits, u32 pass, u32 *rpos, const ShareBufs &b, u64 *wc,
                  cudaStream_t st) {
    const unsigned g = resident_grid((const void *)k_locate_join<COUNT, POW2, D>, 256,
                                     (nhits / JOIN_PASSES + 63) / 64 * 32 + 32);
    if (nhits + (u64)g * 8 * 256 * D + 256 * D >= (1ull << 32)) {   // queue positions are u32
        mb_set_error("locate: %llu hits exceed the walk queue", (unsigned long long)nhits);
        return MB_ERR_ARG;
    }
    const u32 nc = (u32)join_coarse(I.n);
    k_locate_join<COUNT, POW2, D><<<g, 256, nc * sizeof(uint4), st>>>(I, rows, b.idx, b.range, pass, b.wb, b.coarse,
                                                                      nc, b.before, b.nojoin, rpos, b.qhead, wc);
    MB_KCHECK();
    return MB_OK;
}
int launch_join(const DevIndex &I, const u32 *rows, u64 nhits, u32 pass, u32 *rpos, const ShareBufs &b, u64 *wc,
                bool count, u32 depth, cudaStream_t st) {
    const bool pow2 = (I.r & (I.r - 1)) == 0;
    if (count) return pow2 ? launch_join_t<true, true, 1>(I, rows, nhits, pass, rpos, b, wc, st)
                           : launch_join_t<true, false, 1>(I, rows, nhits, pass, rpos, b, wc, st);
    if (!pow2) return launch_join_t<false, false, 1>(I, rows, nhits, pass, rpos, b, wc, st);
    if (depth >= 16) return launch_join_t<false, true, 16>(I, rows, nhits, pass, rpos, b, wc, st);
    if (depth >= 8) return launch_join_t<false, true, 8>(I, rows, nhits, pass, rpos, b, wc, st);
    if (depth >= 4) return launch_join_t<false, true, 4>(I, rows, nhits, pass, rpos, b, wc, st);
    if (depth >= 2) return launch_join_t<false, true, 2>(I, rows, nhits, pass, rpos, b, wc, st);
    return launch_join_t<false, true, 1>(I, rows, nhits, pass, rpos, b, wc, st);
}

size_t share_tmp_bytes(u64 cap, u64 rows_cap) {
    size_t t = radix_tmp_bytes(cap);
    const size_t z[2] = {scan_tmp_bytes(cap), scan_tmp_bytes(JOIN_PASSES * join_tiles(rows_cap) + 1)};
    for (size_t v : z) t = v > t ? v : t;
    return t;
}
// bytes of the per-record arrays (keys, keys_alt, roff: u64; vals, vals_alt, pmax, last: u32)
constexpr size_t SHARE_BYTES_PER_RECORD = 3 * 8 + 4 * 4;

// Locate of the records sm[0, nsm), nsm = min(cap, *nsm_dev): every hit of every record without
// MB_SMEM_OVER_MAX_OCC, written at the record's hit offset (hits_cap bounds every write).  Each
// distinct row is walked once (see the shared-walk kernels); kt, when given, times the walks.
int locate_shared(const DevIndex &I, const mb_smem *sm, u64 cap, const u64 *nsm_dev, const u32 *known, u32 *hits,
                  u64 hits_cap, const ShareBufs &b, u64 *wc, bool count, u32 depth, KTimer *kt, cudaStream_t st) {
    if (cap == 0) return MB_OK;
    const unsigned G = grid_for(cap, 256);
    k_share_flag<<<G, 256, 0, st>>>(sm, cap, nsm_dev, known, hits, hits_cap, b.roff, I.n, b.err);
    MB_KCHECK();
    MB_TRY(scan_exclusive_u64(b.roff, b.roff, cap, b.nwalk, b.tmp, st));
    k_share_compact<<<G, 256, 0, st>>>(sm, cap, nsm_dev, known, b.roff, b.keys, b.vals, I.n);
    MB_KCHECK();
    const BitRange r[1] = {{0, share_key_bits(I.n)}};
    MB_TRY(radix_sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, cap, r, 1, b.tmp, st, b.nwalk));
    u32 *ss = b.vals_alt;   // the sort's scratch, free again
    u64 *sho = b.keys_alt;
    k_share_gather<<<G, 256, 0, st>>>(sm, b.keys, b.vals, cap, b.nwalk, ss, sho, b.pmax);
    MB_KCHECK();
    MB_TRY(scan_inclusive_max_u32(b.pmax, b.pmax, cap, b.tmp, st));
    k_share_mark<<<G, 256, 0, st>>>(b.keys, ss, cap, b.nwalk, b.pmax, b.roff, b.last);
    MB_KCHECK();
    MB_TRY(scan_exclusive_u64(b.roff, b.roff, cap, b.nrows, b.tmp, st));
    MB_TRY(scan_inclusive_max_u32(b.last, b.last, cap, b.tmp, st));
    k_share_rows<<<G, 256, 0, st>>>(b.keys, ss, b.last, b.roff, cap, b.nwalk, b.rows, hits_cap);
    MB_KCHECK();
    u32 *chk = b.checked ? b.err : nullptr;
    const bool aux = b.aux && I.sa_aux;
    if (b.join && b.wb && !chk && !aux) {
        // walk blocks with the marks of the walked rows and their ranks, the rows by pass, then
        // the walks (a walk joins only rows of complete passes)
        const u64 nw = join_words(I.n), nt = join_tiles(hits_cap);   // blocks, partition tiles
        MB_CK(cudaMemsetAsync(b.nojoin, 0, 4, st));
        MB_CK(cudaMemsetAsync(b.qhead, 0, JOIN_PASSES * 4, st));
        k_walk_blocks<<<grid_for(nw, 256), 256, 0, st>>>(I, nw, b.coarse, b.wb);
        MB_KCHECK();
        const unsigned GR = grid_for(hits_cap, 256);
        k_join_mark<<<GR, 256, 0, st>>>(b.rows, b.nrows, hits_cap, b.wb, b.before, b.nojoin);
        MB_KCHECK();
        const unsigned GT = grid_for(nt * 32, 256);
        k_pass_split<false><<<GT, 256, 0, st>>>(b.rows, b.nrows, hits_cap, nt, b.tcnt, b.idx, b.range);
        MB_KCHECK();
        MB_TRY(scan_exclusive_u32(b.tcnt, b.tcnt, JOIN_PASSES * nt, nullptr, b.tmp, st));
        k_pass_split<true><<<GT, 256, 0, st>>>(b.rows, b.nrows, hits_cap, nt, b.tcnt, b.idx, b.range);
        MB_KCHECK();
        if (count) k_join_flag_count<<<1, 32, 0, st>>>(b.nojoin, wc);
        if (kt) kt->start();
        for (u32 p = 0; p < (u32)JOIN_PASSES; ++p) MB_TRY(launch_join(I, b.rows, hits_cap, p, b.rpos, b, wc, count, depth, st));
        if (kt) kt->stop();
    } else {
        DevIndex L = I;   // with MB_LOCATE_AUX the walks stop at the rate-4 samples
        if (aux) {
            L.ssa = I.sa_aux;
            L.r = AUX_RATE;
        }
        if (kt) kt->start();
        MB_TRY(launch_locate(L, b.rows, hits_cap, b.nrows, b.rpos, b.lq, wc, count, depth, chk, st));
        if (kt) kt->stop();
    }
    k_share_copy<<<G, 256, 0, st>>>(b.keys, ss, sho, b.last, b.roff, cap, b.nwalk, b.rpos, hits_cap, hits, hits_cap);
    MB_KCHECK();
    return MB_OK;
}

// The SMEM kernel in the requested shape: work counters, work queue, threads per block.
int launch_smem(const SmemArgs &a, bool count, bool queue, int block, cudaStream_t st) {
    if (count) return launch_smem_t<true, false, 256>(a, st);
    if (queue) {
        if (block == 128) return launch_smem_t<false, true, 128>(a, st);
        if (block == 512) return launch_smem_t<false, true, 512>(a, st);
        return launch_smem_t<false, true, 256>(a, st);
    }
    if (block == 128) return launch_smem_t<false, false, 128>(a, st);
    if (block == 512) return launch_smem_t<false, false, 512>(a, st);
    return launch_smem_t<false, false, 256>(a, st);
}

}  // namespace

// ============================================================================ host entry points
// The seeding pipeline on device inputs (seq, off, mate, and optionally a per-read (l | c << 16));
// out may be host or device.
int mb_seed_device(const mb_index *idx, const u8 *dseq, const u64 *doff, u32 n_reads, const u8 *dmate,
                       const u32 *dlc, u64 o0, u64 o1, const mb_opts *opts, cudaStream_t st, mb_smem *out, u64 cap,
                       u64 *n_out, u64 *n_hits) {
    u32 l, c, max_occ, flags;
    opts_defaults(opts, l, c, max_occ, flags);
    const u32 bs = (flags & MB_BS3) ? 1u : 0u;
    *n_out = 0;
    if (n_hits) *n_hits = 0;
    if (n_reads == 0) return MB_OK;
    const u64 nslots = slots_total(o1 - o0, n_reads);
    DevBuf bslots, bcounts, bsoff, bovf, bmisc, btmp;
    MB_TRY(bslots.alloc(nslots * sizeof(SlotRec), st));
    MB_TRY(bcounts.alloc((size_t)n_reads * 8, st));
    MB_TRY(bsoff.alloc((size_t)n_reads * 8, st));
    MB_TRY(bovf.alloc((size_t)n_reads * 4, st));
    MB_TRY(bmisc.alloc(64, st));
    u64 *dtotal = bmisc.as<u64>(), *dhtotal = bmisc.as<u64>() + 1;
    u32 *dovf_n = (u32 *)(bmisc.as<u64>() + 2), *dqhead = (u32 *)(bmisc.as<u64>() + 3);
    u32 *derr = (u32 *)(bmisc.as<u64>() + 4);
    MB_CK(cudaMemsetAsync(bmisc.p, 0, 64, st));

    const DevIndex I = mb_dev_index(idx);
    const unsigned B = 256;
    const unsigned G = (unsigned)((n_reads + B - 1) / B);
    KTimer kt("smem", st);   // reported after the stream is synchronized below
    const bool kmer = !(flags & MB_NO_KMER) && l >= mb_dev_index(idx).kmer_k;
    {
        const bool count = (flags & MB_COUNT) != 0;
        // with MB_BATCHED the reads are taken from a work queue in read order (no sort here)
        const bool queue = !count && (flags & MB_BATCHED);
        SmemArgs sa{I, (const u8 *)dseq, (const u64 *)doff, n_reads, (const u8 *)dmate, bs, l, c, kmer,
                    bslots.as<SlotRec>(), nslots, bcounts.as<u64>(), bovf.as<u32>(), dovf_n, nullptr,
                    queue ? dqhead : nullptr, count ? mb_work_counter_buf(st) : nullptr, dlc,
                    I.text2 && !(flags & MB_STEP_ONLY)};
        smem_tuning(opts, sa);
        sa.err = derr;
        sa.chk = (flags & MB_CHECKED) ? derr : nullptr;
        const int blk = opts && (opts->block_size == 128 || opts->block_size == 512) ? (int)opts->block_size : 256;
        kt.start();
        MB_TRY(launch_smem(sa, count, queue, blk, st));
        kt.stop();
    }
    MB_TRY(btmp.alloc(scan_tmp_bytes(n_reads), st));
    MB_TRY(scan_exclusive_u64(bcounts.as<u64>(), bsoff.as<u64>(), n_reads, dtotal, btmp.p, st));
    u64 total = 0;
    u32 err = 0;
    MB_CK(cudaMemcpyAsync(&total, dtotal, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaMemcpyAsync(&err, derr, 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (err) {
        mb_set_error("mb_seed_batch: device check failed (0x%x): %s", err,
                     (err & DEVCHK_OFFSETS) ? "read offsets decrease or leave [off[0], off[n_reads]]"
                                            : "an occurrence row outside the text");
        return MB_ERR_DEVICE_CHECK;
    }
    *n_out = total;
    if (total > cap) return MB_ERR_CAPACITY;
    if (total == 0) return MB_OK;

    const bool out_dev = mb_is_device_ptr(out);
    if (!out) {
        mb_set_error("mb_seed_batch: null output");
        return MB_ERR_ARG;
    }
    MB_TRY(mb_check_span(out, total * sizeof(mb_smem), "mb_seed_batch: out"));
    DevBuf bout, bhitc, bhtmp;
    mb_smem *dout = out;
    if (!out_dev) {
        MB_TRY(bout.alloc(total * sizeof(mb_smem), st));
        dout = bout.as<mb_smem>();
    }
    MB_TRY(bhitc.alloc(total * 8, st));
    k_gather<<<G, B, 0, st>>>((const u64 *)doff, n_reads, bslots.as<SlotRec>(), nslots, bcounts.as<u64>(),
                              bsoff.as<u64>(), max_occ, dout, bhitc.as<u64>(), total);
    MB_KCHECK();
    k_smem_overflow<<<resident_grid((const void *)k_smem_overflow, 128, 1ull << 40), 128, 0, st>>>(I, (const u8 *)dseq, (const u64 *)doff, n_reads, (const u8 *)dmate, bs, l,
                                         c, kmer,
                                         bovf.as<u32>(), dovf_n, bsoff.as<u64>(), max_occ, dout, bhitc.as<u64>(),
                                         total, dlc);
    MB_KCHECK();
    MB_TRY(bhtmp.alloc(scan_tmp_bytes(total), st));
    MB_TRY(scan_exclusive_u64(bhitc.as<u64>(), bhitc.as<u64>(), total, dhtotal, bhtmp.p, st));
    k_set_hitoff<<<grid_for(total, 256), 256, 0, st>>>(bhitc.as<u64>(), total, nullptr, dout);
    MB_KCHECK();
    u64 ht = 0;
    MB_CK(cudaMemcpyAsync(&ht, dhtotal, 8, cudaMemcpyDeviceToHost, st));
    if (!out_dev) MB_CK(cudaMemcpyAsync(out, dout, total * sizeof(mb_smem), cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (n_hits) *n_hits = ht;
    return MB_OK;
}

extern "C" int mb_seed_batch(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                             const uint8_t *mate, const mb_opts *opts, void *stream, mb_smem *out, uint64_t cap,
                             uint64_t *n_out, uint64_t *n_hits) {
    if (!idx || !off || !n_out || (n_reads > 0 && !seq)) {
        mb_set_error("mb_seed_batch: null argument");
        return MB_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    *n_out = 0;
    if (n_hits) *n_hits = 0;
    if (n_reads == 0) return MB_OK;

    // offsets to the host to size the inputs and scratch
    DevBuf boff, bseq, bmate;
    const void *doff = nullptr, *dseq = nullptr, *dmate = nullptr;
    u64 o0 = 0, o1 = 0;
    MB_TRY(mb_check_span(off, (size_t)(n_reads + 1) * 8, "mb_seed_batch: off"));
    MB_CK(cudaMemcpyAsync(&o0, off, 8, cudaMemcpyDefault, st));
    MB_CK(cudaMemcpyAsync(&o1, off + n_reads, 8, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    if (o1 < o0) {
        mb_set_error("mb_seed_batch: offsets decrease");
        return MB_ERR_ARG;
    }
    MB_TRY(mb_check_span(seq + o0, o1 - o0, "mb_seed_batch: seq[off[0], off[n_reads])"));
    if (mate) MB_TRY(mb_check_span(mate, n_reads, "mb_seed_batch: mate"));
    MB_TRY(mb_stage_in(off, (size_t)(n_reads + 1) * 8, st, boff, &doff));
    // a host `seq` is staged from off[0]; device pointers are used as given
    if (mb_is_device_ptr(seq)) dseq = seq;
    else {
        MB_TRY(bseq.alloc(o1 - o0 + 1, st));
        MB_CK(cudaMemcpyAsync(bseq.as<u8>() + 0, seq + o0, o1 - o0, cudaMemcpyHostToDevice, st));
        dseq = bseq.as<u8>() - o0;
    }
    if (mate) MB_TRY(mb_stage_in(mate, n_reads, st, bmate, &dmate));

    return mb_seed_device(idx, (const u8 *)dseq, (const u64 *)doff, n_reads, (const u8 *)dmate, nullptr, o0, o1, opts,
                       st, out, cap, n_out, n_hits);
}

// The shared-walk workspace for n_smem records and total hits on an index of n rows (with the
// arrays of the walks that join unless `join` is false), carved from one stream-ordered allocation.
static int share_alloc(DevBuf &bw, u64 n_smem, u64 total, u64 n, bool join, cudaStream_t st, ShareBufs &b) {
    const size_t rec_bytes = (size_t)n_smem * SHARE_BYTES_PER_RECORD, row_bytes = (size_t)total * 8;
    const size_t tmp = share_tmp_bytes(n_smem, total), jb = join ? join_bytes(n, total) : 0;
    MB_TRY(bw.alloc(rec_bytes + row_bytes + 16 + tmp + jb + 15 * 256, st));
    char *m = (char *)bw.p;
    auto take = [&](size_t bytes) { void *p = m; m += (bytes + 255) & ~(size_t)255; return p; };
    b.keys = (u64 *)take(n_smem * 8);
    b.keys_alt = (u64 *)take(n_smem * 8);
    b.roff = (u64 *)take(n_smem * 8);
    b.vals = (u32 *)take(n_smem * 4);
    b.vals_alt = (u32 *)take(n_smem * 4);
    b.pmax = (u32 *)take(n_smem * 4);
    b.last = (u32 *)take(n_smem * 4);
    b.rows = (u32 *)take(total * 4);
    b.rpos = (u32 *)take(total * 4);
    b.nrows = (u64 *)take(8);
    b.nwalk = (u64 *)take(8);
    b.err = (u32 *)take(8);
    b.lq = (u32 *)take(8);
    b.tmp = take(tmp);
    b.join = join;
    if (join) {   // the order and sizes of join_bytes
        b.wb = (WalkBlk *)take(join_words(n) * sizeof(WalkBlk));
        b.coarse = (uint4 *)take(join_coarse(n) * 16);
        b.before = (u32 *)take(join_words(n) * 4);
        b.nojoin = (u32 *)take(8);
        b.tcnt = (u32 *)take(JOIN_PASSES * join_tiles(total) * 4 + 4);
        b.idx = (u32 *)take(total * 4);
        b.range = (u64 *)take((JOIN_PASSES + 1) * 8);
        b.qhead = (u32 *)take(JOIN_PASSES * 4);
    }
    MB_CK(cudaMemsetAsync(b.err, 0, 8, st));
    return MB_OK;
}

int mb_locate_records(const mb_index *idx, const mb_smem *sm, u64 n_smem, const u32 *known, u32 *hits, u64 n_hits,
                      u32 depth, bool join, bool aux, cudaStream_t st) {
    if (n_smem == 0 || n_hits == 0) return MB_OK;
    DevBuf bw;
    ShareBufs b;
    const DevIndex I = mb_dev_index(idx);
    MB_TRY(share_alloc(bw, n_smem, n_hits, I.n, join && !aux && n_hits > 1, st, b));
    b.aux = aux;
    return locate_shared(I, sm, n_smem, nullptr, known, hits, n_hits, b, nullptr, false, depth, nullptr, st);
}

extern "C" int mb_locate(const mb_index *idx, const mb_smem *smem, uint64_t n_smem, const mb_opts *opts,
                         void *stream, uint32_t *hits, uint64_t cap, uint64_t *n_hits) {
    if (!idx || !n_hits || (n_smem && !smem)) {
        mb_set_error("mb_locate: null argument");
        return MB_ERR_ARG;
    }
    *n_hits = 0;
    if (n_smem == 0) return MB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf bsm, bhits;
    const void *dsm = nullptr;
    MB_TRY(mb_check_span(smem, n_smem * sizeof(mb_smem), "mb_locate: smem"));
    MB_TRY(mb_stage_in(smem, n_smem * sizeof(mb_smem), st, bsm, &dsm));
    mb_smem last;
    MB_CK(cudaMemcpyAsync(&last, (const mb_smem *)dsm + n_smem - 1, sizeof last, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    u64 total = last.hit_off + ((last.flags & MB_SMEM_OVER_MAX_OCC) ? 0 : last.s);
    *n_hits = total;
    if (total > cap) return MB_ERR_CAPACITY;
    if (total == 0) return MB_OK;
    if (!hits) return MB_ERR_ARG;
    MB_TRY(mb_check_span(hits, total * 4, "mb_locate: hits"));
    u32 *dh = hits;
    const bool hdev = mb_is_device_ptr(hits);
    if (!hdev) {
        MB_TRY(bhits.alloc(total * 4, st));
        dh = bhits.as<u32>();
    }
    const DevIndex I = mb_dev_index(idx);
    const bool count = opts && (opts->flags & MB_COUNT);
    DevBuf bw;
    ShareBufs b;
    MB_TRY(share_alloc(bw, n_smem, total, I.n,
                       opts && (opts->flags & MB_LOCATE_JOIN) && !(opts->flags & (MB_CHECKED | MB_LOCATE_AUX)), st,
                       b));
    b.aux = opts && (opts->flags & MB_LOCATE_AUX);
    b.checked = opts && (opts->flags & MB_CHECKED);
    u64 *wc = count ? mb_work_counter_buf(st) : nullptr;
    KTimer kt("locate", st);
    MB_TRY(locate_shared(I, (const mb_smem *)dsm, n_smem, nullptr, nullptr, dh, total, b, wc, count,
                         opts ? opts->prefetch_depth : 0, &kt, st));
    u32 err = 0;
    MB_CK(cudaMemcpyAsync(&err, b.err, 4, cudaMemcpyDeviceToHost, st));
    if (!hdev) MB_CK(cudaMemcpyAsync(hits, dh, total * 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (err) {
        mb_set_error("mb_locate: device check failed (0x%x): %s", err,
                     (err & DEVCHK_RECORD) ? "a record's rows [k, k+s) leave the text" : "a row outside the text");
        return MB_ERR_DEVICE_CHECK;
    }
    return MB_OK;
}

extern "C" int mb_bs_filter(const mb_index *idx, const mb_smem *smem, uint64_t n_smem, const uint8_t *mate,
                            const uint32_t *hits, uint64_t n_hits, void *stream, uint8_t *keep) {
    if (!idx || (n_hits && (!smem || !hits || !keep))) return MB_ERR_ARG;
    if (n_hits == 0) return MB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf bsm, bmate, bhits, bkeep;
    const void *dsm = nullptr, *dmate = nullptr, *dhits = nullptr;
    MB_TRY(mb_stage_in(smem, n_smem * sizeof(mb_smem), st, bsm, &dsm));
    if (mate) {
        mb_smem last;
        MB_CK(cudaMemcpyAsync(&last, (const mb_smem *)dsm + n_smem - 1, sizeof last, cudaMemcpyDeviceToHost, st));
        MB_CK(cudaStreamSynchronize(st));
        MB_TRY(mb_stage_in(mate, (size_t)last.read + 1, st, bmate, &dmate));
    }
    MB_TRY(mb_stage_in(hits, n_hits * 4, st, bhits, &dhits));
    u8 *dk = keep;
    const bool kdev = mb_is_device_ptr(keep);
    if (!kdev) {
        MB_TRY(bkeep.alloc(n_hits, st));
        dk = bkeep.as<u8>();
    }
    u64 M = 0, n = 0, prim = 0;
    mb_index_info(idx, &n, &prim, &M);
    // the 3-base index holds four copies of |R| = M/2 bases
    u64 quarter = M / 2;
    k_bs_filter<<<grid_for(n_hits, 256), 256, 0, st>>>((const mb_smem *)dsm, n_smem, (const u8 *)dmate,
                                                       (const u32 *)dhits, n_hits, quarter, dk);
    MB_KCHECK();
    if (!kdev) MB_CK(cudaMemcpyAsync(keep, dk, n_hits, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    return MB_OK;
}

// ============================================================================ no-allocation variant
// mb_seed_batch_noalloc is for callers that cannot allocate device memory: a host process whose
// device memory is already reserved in full by another allocator (a framework's caching
// allocator, a serving runtime that pre-reserves HBM), or a latency-critical caller for which a
// cudaMalloc / cudaFree (which may synchronize the device) is not acceptable.  Its scratch is
// the fixed array below; the caller still provides the inputs and the output records.
//
// The array is part of this library's device image: every GPU on which the library is loaded
// holds these MB_NOALLOC_SCRATCH_BYTES until the process exits.  All calls share it and it keeps
// the contents of the last call, so calls whose work overlaps on the GPU (other streams or
// threads) race; calls on one stream are ordered.
#define MB_NOALLOC_SCRATCH_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[MB_NOALLOC_SCRATCH_BYTES];

#include <mutex>

namespace {
constexpr int NOALLOC_MAX_DEV = 128;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEV] = {};

// Device address of the scratch array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device, with that device
// current, and cached.  The first call on a device does this set-up; make that first call before
// any stream capture.
int noalloc_scratch(unsigned char **p) {
    int d = 0;
    MB_CK(cudaGetDevice(&d));
    if (d < 0 || d >= NOALLOC_MAX_DEV) {
        mb_set_error("mb_seed_batch_noalloc: device ordinal %d out of range", d);
        return MB_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[d]) {
        void *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        if (e != cudaSuccess || !q) {
            mb_set_error("mb_seed_batch_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return MB_ERR_CUDA;
        }
        g_noalloc_ptr[d] = q;
    }
    *p = (unsigned char *)g_noalloc_ptr[d];
    return MB_OK;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

extern "C" int mb_seed_batch_noalloc(const mb_index *idx, const uint8_t *seq, const uint64_t *off,
                                     uint32_t n_reads, const uint8_t *mate, const mb_opts *opts, void *stream,
                                     mb_smem *out, uint64_t cap, uint64_t *n_out, uint64_t *n_hits) {
    if (!idx || !off || !n_out || (n_reads > 0 && (!seq || !out))) {
        mb_set_error("mb_seed_batch_noalloc: null argument");
        return MB_ERR_ARG;
    }
    *n_out = 0;
    if (n_hits) *n_hits = 0;
    if (n_reads == 0) return MB_OK;
    if (!mb_is_device_ptr(seq) || !mb_is_device_ptr(off) || !mb_is_device_ptr(out) ||
        (mate && !mb_is_device_ptr(mate))) {
        mb_set_error("mb_seed_batch_noalloc: seq, off, mate and out must be device pointers");
        return MB_ERR_ARG;
    }
    u32 l, c, max_occ, flags;
    opts_defaults(opts, l, c, max_occ, flags);
    const u32 bs = (flags & MB_BS3) ? 1u : 0u;
    cudaStream_t st = (cudaStream_t)stream;
    u64 o0 = 0, o1 = 0;
    MB_TRY(mb_check_span(off, (size_t)(n_reads + 1) * 8, "mb_seed_batch_noalloc: off"));
    MB_CK(cudaMemcpyAsync(&o0, off, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaMemcpyAsync(&o1, off + n_reads, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (o1 < o0) {
        mb_set_error("mb_seed_batch_noalloc: offsets decrease");
        return MB_ERR_ARG;
    }
    MB_TRY(mb_check_span(seq + o0, o1 - o0, "mb_seed_batch_noalloc: seq[off[0], off[n_reads])"));
    if (mate) MB_TRY(mb_check_span(mate, n_reads, "mb_seed_batch_noalloc: mate"));
    // scratch layout: [totals][counts][soff][overflow list][scan tmp][slots][hit counts][scan tmp]
    const size_t nr = n_reads;
    const size_t nslots = slots_total(o1 - o0, nr);
    const size_t o_cnt = 256, o_soff = o_cnt + al256(nr * 8), o_ovf = o_soff + al256(nr * 8);
    const size_t o_tmp = o_ovf + al256(nr * 4), o_slots = o_tmp + al256(scan_tmp_bytes(nr));
    const size_t fixed = o_slots + al256(nslots * sizeof(SlotRec));
    if (fixed > MB_NOALLOC_SCRATCH_BYTES) {
        mb_set_error("mb_seed_batch_noalloc: batch of %zu reads / %llu bases needs %zu bytes of scratch, "
                     "more than the fixed %llu; split the batch",
                     nr, (unsigned long long)(o1 - o0), fixed, (unsigned long long)MB_NOALLOC_SCRATCH_BYTES);
        return MB_ERR_ARG;
    }
    unsigned char *S = nullptr;
    MB_TRY(noalloc_scratch(&S));
    u64 *dtotal = (u64 *)S, *dhtotal = (u64 *)S + 1;
    u32 *dovf_n = (u32 *)((u64 *)S + 2), *derr = (u32 *)((u64 *)S + 3);
    u64 *counts = (u64 *)(S + o_cnt), *soff = (u64 *)(S + o_soff);
    u32 *ovf = (u32 *)(S + o_ovf);
    SlotRec *slots = (SlotRec *)(S + o_slots);
    MB_CK(cudaMemsetAsync(S, 0, 256, st));   // totals and the overflow count start at zero

    const DevIndex I = mb_dev_index(idx);
    const unsigned B = 256, G = (unsigned)((nr + B - 1) / B);
    const bool kmer = !(flags & MB_NO_KMER) && l >= I.kmer_k;
    {
        SmemArgs sa{I, seq, off, n_reads, mate, bs, l, c, kmer, slots, nslots, counts, ovf, dovf_n, nullptr, nullptr,
                    nullptr, nullptr, I.text2 && !(flags & MB_STEP_ONLY)};
        smem_tuning(opts, sa);
        sa.err = derr;
        sa.chk = (flags & MB_CHECKED) ? derr : nullptr;
        MB_TRY(launch_smem(sa, false, false, 256, st));
    }
    MB_TRY(scan_exclusive_u64(counts, soff, nr, dtotal, S + o_tmp, st));
    u64 total = 0;
    u32 err = 0;
    MB_CK(cudaMemcpyAsync(&total, dtotal, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaMemcpyAsync(&err, derr, 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (err) {
        mb_set_error("mb_seed_batch_noalloc: device check failed (0x%x)", err);
        return MB_ERR_DEVICE_CHECK;
    }
    *n_out = total;
    if (total > cap) return MB_ERR_CAPACITY;
    if (total == 0) return MB_OK;
    MB_TRY(mb_check_span(out, total * sizeof(mb_smem), "mb_seed_batch_noalloc: out"));
    const size_t o_hitc = fixed, o_htmp = o_hitc + al256(total * 8);
    const size_t need = o_htmp + al256(scan_tmp_bytes(total));
    if (need > MB_NOALLOC_SCRATCH_BYTES) {
        mb_set_error("mb_seed_batch_noalloc: %llu SMEMs need %zu bytes of scratch, more than the fixed %llu; "
                     "split the batch",
                     (unsigned long long)total, need, (unsigned long long)MB_NOALLOC_SCRATCH_BYTES);
        *n_out = 0;
        return MB_ERR_ARG;
    }
    u64 *hitc = (u64 *)(S + o_hitc);
    k_gather<<<G, B, 0, st>>>(off, n_reads, slots, nslots, counts, soff, max_occ, out, hitc, total);
    MB_KCHECK();
    k_smem_overflow<<<resident_grid((const void *)k_smem_overflow, 128, 1ull << 40), 128, 0, st>>>(I, seq, off, n_reads, mate, bs, l, c, kmer, ovf, dovf_n, soff, max_occ, out,
                                         hitc, total, nullptr);
    MB_KCHECK();
    MB_TRY(scan_exclusive_u64(hitc, hitc, total, dhtotal, S + o_htmp, st));
    k_set_hitoff<<<grid_for(total, 256), 256, 0, st>>>(hitc, total, nullptr, out);
    MB_KCHECK();
    u64 ht = 0;
    MB_CK(cudaMemcpyAsync(&ht, dhtotal, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (n_hits) *n_hits = ht;
    return MB_OK;
}

// ============================================================================ batched form: plans
struct mb_plan {
    const mb_index *idx = nullptr;
    u32 l = 19, c = 1, max_occ = 500, flags = 0;
    bool kmer = true, queue = false;
    int block = 256;
    u32 depth = 1;   // walks per lane in locate
    bool split = true;   // SMEM kernel form and tuning
    SmemTuning tune = {SMEM_BURST, SMEM_WAIT, 32};
    u32 warps = 0;
    u32 max_reads = 0;
    u64 max_bases = 0, max_smem = 0, max_hits = 0, nslots = 0;
    void *mem = nullptr;
    SlotRec *slots = nullptr;
    u64 *counts = nullptr, *soff = nullptr, *misc = nullptr, *hitc = nullptr;
    u32 *ovf = nullptr, *rows = nullptr, *hits = nullptr;
    u32 *known = nullptr;   // per record: the hit position found while seeding, or NOPOS
    ShareBufs share;        // shared-walk locate: per-record arrays, positions of the walked rows
    mb_smem *out = nullptr;
    void *tmp = nullptr;
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    u64 graph_kernels = 0;   // kernel nodes of the captured graph
};

size_t mb_plan_bytes(const mb_plan *p) { return p ? p->bytes : 0; }
// The plan's device error word: the upper half of misc[2] (its lower half counts the reads that
// overflow their slots), so that misc[0..2] carry both counts and the error word in one copy.
static u32 *plan_err(const mb_plan *p) { return (u32 *)(p->misc + 2) + 1; }
int mb_plan_counts_async(mb_plan *p, u64 *host_counts, cudaStream_t st) {
    MB_CK(cudaMemcpyAsync(host_counts, p->misc, 24, cudaMemcpyDeviceToHost, st));
    return MB_OK;
}
void mb_plan_arrays(const mb_plan *p, const mb_smem **smem, const u32 **hits, u64 *max_smem, u64 *max_hits) {
    *smem = p->out;
    *hits = p->hits;
    *max_smem = p->max_smem;
    *max_hits = p->max_hits;
}

// Device workspace of a plan, one entry per array (in the order mb_plan_create lays them out).
constexpr int PLAN_ARRAYS = 27;
// A plan locates with walks that join (their arrays sized by the index's n rows) when the options
// say MB_LOCATE_JOIN without MB_CHECKED or MB_LOCATE_AUX and the plan holds hits to locate (not a
// seeding-only plan).
static bool plan_joins(const mb_opts *opts, u64 max_hits) {
    return opts && (opts->flags & MB_LOCATE_JOIN) && !(opts->flags & (MB_CHECKED | MB_LOCATE_AUX)) && max_hits > 1;
}
static void plan_sizes(const mb_opts *opts, u64 n, u32 max_reads, u64 max_bases, u64 max_smem, u64 max_hits,
                       size_t sizes[PLAN_ARRAYS]) {
    const size_t nr = max_reads, ms = max_smem ? max_smem : 1, mh = max_hits ? max_hits : 1;
    size_t tb = scan_tmp_bytes(nr > ms ? nr : ms);
    const size_t sb = share_tmp_bytes(ms, mh);
    if (sb > tb) tb = sb;
    const bool join = plan_joins(opts, max_hits);
    const size_t nw = join ? join_words(n) : 0, nc = join ? join_coarse(n) : 0, nt = join ? join_tiles(mh) : 0;
    const size_t z[PLAN_ARRAYS] = {slots_total(max_bases, max_reads) * sizeof(SlotRec), nr * 8, nr * 8, 256, ms * 8,
                                   nr * 4, mh * 4, mh * 4, ms * sizeof(mb_smem), tb, ms * 4,
                                   ms * 8, ms * 8, ms * 8, ms * 4, ms * 4, ms * 4, ms * 4, mh * 4,
                                   nw * sizeof(WalkBlk), nc * 16, nw * 4, join ? 8u : 0u,
                                   join ? JOIN_PASSES * nt * 4 + 4 : 0, join ? mh * 4 : 0,
                                   join ? (size_t)(JOIN_PASSES + 1) * 8 : 0, join ? (size_t)JOIN_PASSES * 4 : 0};
    for (int i = 0; i < PLAN_ARRAYS; ++i) sizes[i] = z[i];
}

size_t mb_plan_workspace_bytes(const mb_opts *opts, u64 n, u32 max_reads, u64 max_bases, u64 max_smem,
                               u64 max_hits) {
    size_t sizes[PLAN_ARRAYS], total = 0;
    plan_sizes(opts, n, max_reads, max_bases, max_smem, max_hits, sizes);
    for (size_t z : sizes) total += align_up(z);
    return total;
}

extern "C" int mb_plan_create(const mb_index *idx, const mb_opts *opts, uint32_t max_reads, uint64_t max_bases,
                              uint64_t max_smem, uint64_t max_hits, mb_plan **out) {
    if (!idx || !out || max_reads == 0) return MB_ERR_ARG;
    *out = nullptr;
    mb_plan *P = new mb_plan;
    P->idx = idx;
    opts_defaults(opts, P->l, P->c, P->max_occ, P->flags);
    P->kmer = !(P->flags & MB_NO_KMER) && P->l >= mb_dev_index(idx).kmer_k;
    P->queue = (P->flags & MB_BATCHED) != 0;
    P->block = opts && (opts->block_size == 128 || opts->block_size == 512) ? (int)opts->block_size : 256;
    const u32 dq = opts ? opts->prefetch_depth : 0;
    P->depth = dq >= 16 ? 16u : (dq >= 8 ? 8u : (dq >= 4 ? 4u : (dq >= 2 ? 2u : 1u)));
    {
        SmemArgs t{};
        smem_tuning(opts, t);
        P->split = t.split;
        P->tune = t.tune;
        P->warps = t.warps;
    }
    P->max_reads = max_reads;
    P->max_bases = max_bases;
    P->max_smem = max_smem ? max_smem : 1;
    P->max_hits = max_hits ? max_hits : 1;
    P->nslots = slots_total(max_bases, max_reads);
    size_t sizes[PLAN_ARRAYS];
    const u64 n_rows = mb_dev_index(idx).n;
    plan_sizes(opts, n_rows, max_reads, max_bases, max_smem, max_hits, sizes);
    size_t total = 0;
    for (size_t z : sizes) total += align_up(z);
    if (cudaMalloc(&P->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        mb_set_error("mb_plan_create: cannot allocate %zu bytes of device workspace", total);
        return MB_ERR_NOMEM;
    }
    P->bytes = total;
    char *m = (char *)P->mem;
    void **ptrs[PLAN_ARRAYS] = {(void **)&P->slots, (void **)&P->counts, (void **)&P->soff, (void **)&P->misc,
                                (void **)&P->hitc, (void **)&P->ovf, (void **)&P->rows, (void **)&P->hits,
                                (void **)&P->out, (void **)&P->tmp, (void **)&P->known, (void **)&P->share.keys,
                                (void **)&P->share.keys_alt, (void **)&P->share.roff, (void **)&P->share.vals,
                                (void **)&P->share.vals_alt, (void **)&P->share.pmax, (void **)&P->share.last,
                                (void **)&P->share.rpos, (void **)&P->share.wb, (void **)&P->share.coarse,
                                (void **)&P->share.before, (void **)&P->share.nojoin, (void **)&P->share.tcnt,
                                (void **)&P->share.idx, (void **)&P->share.range, (void **)&P->share.qhead};
    for (int i = 0; i < PLAN_ARRAYS; ++i) {
        *ptrs[i] = sizes[i] ? (void *)m : nullptr;
        m += align_up(sizes[i]);
    }
    P->share.rows = P->rows;
    P->share.nrows = P->misc + 4;
    P->share.nwalk = P->misc + 5;
    P->share.tmp = P->tmp;
    P->share.err = plan_err(P);
    P->share.lq = (u32 *)(P->misc + 6);
    P->share.checked = (P->flags & MB_CHECKED) != 0;
    P->share.join = plan_joins(opts, max_hits);
    P->share.aux = (P->flags & MB_LOCATE_AUX) != 0;
    *out = P;
    return MB_OK;
}

extern "C" void mb_plan_free(mb_plan *P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->mem) cudaFree(P->mem);
    delete P;
}

// Seeding of the plan's batch up to the records with their hit offsets (no locate).
static int plan_seed(mb_plan *P, const uint8_t *seq, const uint64_t *off, uint32_t n_reads, const uint8_t *mate,
                     cudaStream_t st) {
    if (!P || (n_reads && (!seq || !off))) return MB_ERR_ARG;
    if (n_reads > P->max_reads) {
        mb_set_error("mb_plan_run: %u reads exceed the plan's %u", n_reads, P->max_reads);
        return MB_ERR_ARG;
    }
    MB_CK(cudaMemsetAsync(P->misc, 0, 256, st));
    if (n_reads == 0) return MB_OK;
    const DevIndex I = mb_dev_index(P->idx);
    const u32 bs = (P->flags & MB_BS3) ? 1u : 0u;
    u64 *n_smem = P->misc, *n_hits = P->misc + 1;
    u32 *ovf_n = (u32 *)(P->misc + 2), *qhead = (u32 *)(P->misc + 3), *err = plan_err(P);
    MB_CK(cudaMemsetAsync(P->hitc, 0, P->max_smem * 8, st));   // zero tail for the fixed-length scan
    // with the work queue the reads are handed out in read order: ordering them by decreasing
    // length (tried: a sort before the launch) made the mixed-length batch 2.4 ms slower
    const u32 *perm = nullptr;
    SmemArgs sa{I, seq, off, n_reads, mate, bs, P->l, P->c, P->kmer, P->slots, P->nslots, P->counts, P->ovf, ovf_n,
                perm, qhead, nullptr, nullptr, I.text2 && !(P->flags & MB_STEP_ONLY)};
    sa.split = P->split;
    sa.tune = P->tune;
    sa.warps = P->warps;
    sa.err = err;
    sa.chk = (P->flags & MB_CHECKED) ? err : nullptr;
    MB_TRY(launch_smem(sa, false, P->queue, P->block, st));
    MB_TRY(scan_exclusive_u64(P->counts, P->soff, n_reads, n_smem, P->tmp, st));
    const unsigned G = (unsigned)((n_reads + 255) / 256);
    k_gather<<<G, 256, 0, st>>>(off, n_reads, P->slots, P->nslots, P->counts, P->soff, P->max_occ, P->out, P->hitc,
                                P->max_smem, P->known);
    MB_KCHECK();
    k_smem_overflow<<<resident_grid((const void *)k_smem_overflow, 128, 1ull << 40), 128, 0, st>>>(I, seq, off, n_reads, mate, bs, P->l, P->c, P->kmer, P->ovf, ovf_n, P->soff,
                                         P->max_occ, P->out, P->hitc, P->max_smem, nullptr, P->known);
    MB_KCHECK();
    MB_TRY(scan_exclusive_u64(P->hitc, P->hitc, P->max_smem, n_hits, P->tmp, st));
    k_set_hitoff<<<grid_for(P->max_smem, 256), 256, 0, st>>>(P->hitc, P->max_smem, n_smem, P->out);
    MB_KCHECK();
    return MB_OK;
}

int mb_plan_run_seed(mb_plan *P, const uint8_t *seq, const uint64_t *off, uint32_t n_reads, const uint8_t *mate,
                     cudaStream_t st) {
    return plan_seed(P, seq, off, n_reads, mate, st);
}
const u32 *mb_plan_known(const mb_plan *P) { return P ? P->known : nullptr; }

// The whole stage on `stream`, with no host synchronization and no allocation.
extern "C" int mb_plan_run(mb_plan *P, const uint8_t *seq, const uint64_t *off, uint32_t n_reads, const uint8_t *mate,
                           void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    MB_TRY(plan_seed(P, seq, off, n_reads, mate, st));
    if (n_reads == 0) return MB_OK;
    MB_TRY(locate_shared(mb_dev_index(P->idx), P->out, P->max_smem, P->misc, P->known, P->hits, P->max_hits,
                         P->share, nullptr, false, P->depth, nullptr, st));
    return MB_OK;
}

extern "C" int mb_plan_result(mb_plan *P, void *stream, const mb_smem **smem, uint64_t *n_smem, const uint32_t **hits,
                              uint64_t *n_hits) {
    if (!P) return MB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    u64 v[3] = {0, 0, 0};
    MB_CK(cudaMemcpyAsync(v, P->misc, 24, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (v[2] >> 32) {
        mb_set_error("mb_plan_result: device check failed (0x%x)", (unsigned)(v[2] >> 32));
        return MB_ERR_DEVICE_CHECK;
    }
    if (n_smem) *n_smem = v[0];
    if (n_hits) *n_hits = v[1];
    if (smem) *smem = P->out;
    if (hits) *hits = P->hits;
    if (v[0] > P->max_smem || v[1] > P->max_hits) {
        mb_set_error("mb_plan_result: %llu SMEMs / %llu hits exceed the plan's %llu / %llu",
                     (unsigned long long)v[0], (unsigned long long)v[1], (unsigned long long)P->max_smem,
                     (unsigned long long)P->max_hits);
        return MB_ERR_CAPACITY;
    }
    return MB_OK;
}

extern "C" int mb_plan_copy(mb_plan *P, void *stream, mb_smem *out, uint64_t cap, uint32_t *hits, uint64_t hits_cap) {
    if (!P) return MB_ERR_ARG;
    u64 ns = 0, nh = 0;
    const mb_smem *sp = nullptr;
    const uint32_t *hp = nullptr;
    MB_TRY(mb_plan_result(P, stream, &sp, &ns, &hp, &nh));
    if ((out && ns > cap) || (hits && nh > hits_cap)) return MB_ERR_CAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    if (out && ns) MB_CK(cudaMemcpyAsync(out, sp, ns * sizeof(mb_smem), cudaMemcpyDefault, st));
    if (hits && nh) MB_CK(cudaMemcpyAsync(hits, hp, nh * 4, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    return MB_OK;
}

extern "C" int mb_plan_capture(mb_plan *P, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                               const uint8_t *mate) {
    if (!P) return MB_ERR_ARG;
    cudaStream_t s;
    MB_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (P->exec) { cudaGraphExecDestroy(P->exec); P->exec = nullptr; }
    if (P->graph) { cudaGraphDestroy(P->graph); P->graph = nullptr; }
    int rc = MB_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MB_ERR_CUDA;
    else {
        rc = mb_plan_run(P, seq, off, n_reads, mate, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc == MB_OK && e != cudaSuccess) rc = MB_ERR_CUDA;
        if (rc == MB_OK && cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) rc = MB_ERR_CUDA;
        if (rc == MB_OK) {
            P->graph = g;
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
            P->graph_kernels = 0;
            for (size_t i = 0; i < nn; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    ++P->graph_kernels;
            }
        }
        else if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(s);
    if (rc != MB_OK) mb_set_error("mb_plan_capture: graph capture failed");
    return rc;
}

extern "C" int mb_plan_replay(mb_plan *P, void *stream) {
    if (!P || !P->exec) return MB_ERR_ARG;
    MB_CK(cudaGraphLaunch(P->exec, (cudaStream_t)stream));
    for (u64 i = 0; i < P->graph_kernels; ++i) mb_count_launch();   // the kernels the graph runs
    return MB_OK;
}

// Times launch shapes on this batch (all give the same output; tests check that), in stages:
// (1) the SMEM kernel's shape, over threads per block {128, 256, 512} x work queue off/on x the
// kernel form (the one-loop form, and the split form with memory steps between service passes
// {2, 4, 8, 16} x lanes out of the loop that call a pass early {4, 8, 16}), with 16 plain locate
// walks per lane; (2) for a split-form winner, reads per warp {1, 2, 4, 8, 16}; (3) with the best
// SMEM shape, locate walks per lane {1, 2, 4, 8} plain and {1, 2, 4, 8, 16} with walks that join
// (MB_LOCATE_JOIN).  Each point is the
// best of two timed runs of mb_plan_run after one untimed run.  Every point tried is written to
// points / points_ms when given (up to cap; *n_points receives the number tried).
static int autotune_impl(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                         const mb_opts *opts, cudaStream_t st, mb_opts *best, double *best_ms, mb_opts *points,
                         double *points_ms, uint32_t cap, uint32_t *n_points) {
    if (!idx || !best || !seq || !off || n_reads == 0) return MB_ERR_ARG;
    // sizes from one run of the allocating path
    u64 n_smem = 0, n_hits = 0;
    {
        mb_opts o = opts ? *opts : mb_opts{};
        DevBuf tmp;
        int rc = mb_seed_batch(idx, seq, off, n_reads, nullptr, &o, st, nullptr, 0, &n_smem, &n_hits);
        if (rc != MB_OK && rc != MB_ERR_CAPACITY) return rc;
        MB_TRY(tmp.alloc(n_smem * sizeof(mb_smem) + 64, st));
        MB_TRY(mb_seed_batch(idx, seq, off, n_reads, nullptr, &o, st, tmp.as<mb_smem>(), n_smem, &n_smem, &n_hits));
    }
    u64 o0 = 0, o1 = 0;
    MB_CK(cudaMemcpyAsync(&o0, off, 8, cudaMemcpyDefault, st));
    MB_CK(cudaMemcpyAsync(&o1, off + n_reads, 8, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    cudaEvent_t a, b;
    MB_CK(cudaEventCreate(&a));
    MB_CK(cudaEventCreate(&b));
    u32 np = 0;
    double bms = 1e30;
    mb_opts bo = opts ? *opts : mb_opts{};
    auto time_point = [&](const mb_opts &o) -> int {
        mb_plan *P = nullptr;
        int rc = mb_plan_create(idx, &o, n_reads, o1 - o0, n_smem, n_hits, &P);
        if (rc != MB_OK) return rc;
        double t_best = 1e30;
        for (int rep = 0; rep < 3 && rc == MB_OK; ++rep) {
            cudaEventRecord(a, st);
            rc = mb_plan_run(P, seq, off, n_reads, nullptr, st);
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess) rc = MB_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < t_best) t_best = ms;   // the first run warms up
        }
        mb_plan_free(P);
        if (rc != MB_OK) return rc;
        if (points && np < cap) {
            points[np] = o;
            if (points_ms) points_ms[np] = t_best;
        }
        ++np;
        if (t_best < bms) {
            bms = t_best;
            bo = o;
        }
        return MB_OK;
    };
    int rc = MB_OK;
    const int blocks[3] = {128, 256, 512};
    const u32 bursts[4] = {2, 4, 8, 16}, waits[3] = {4, 8, 16};
    for (int q = 0; q < 2 && rc == MB_OK; ++q)
        for (int bi = 0; bi < 3 && rc == MB_OK; ++bi)
            for (int f = -1; f < 12 && rc == MB_OK; ++f) {
                mb_opts o = opts ? *opts : mb_opts{};
                o.flags = (o.flags & ~(MB_BATCHED | MB_SMEM_ONE_LOOP | MB_LOCATE_JOIN)) | (q ? MB_BATCHED : 0u);
                o.smem_reads_per_warp = 0;
                o.block_size = (u32)blocks[bi];
                o.prefetch_depth = 16;
                if (f < 0) {
                    o.flags |= MB_SMEM_ONE_LOOP;
                    o.smem_burst = o.smem_wait = 0;
                } else {
                    o.smem_burst = bursts[f / 3];
                    o.smem_wait = waits[f % 3];
                }
                rc = time_point(o);
            }
    // reads per warp below 32 (lanes left idle) with the best SMEM shape
    for (u32 rpw = 1; rpw <= 16 && rc == MB_OK && !(bo.flags & MB_SMEM_ONE_LOOP); rpw *= 2) {
        mb_opts o = bo;
        o.smem_reads_per_warp = rpw;
        rc = time_point(o);
    }
    const mb_opts smem_best = bo;
    for (int join = 0; join < 2; ++join)
        for (u32 dep = 1; dep <= (join ? 16u : 8u) && rc == MB_OK; dep *= 2) {
            mb_opts o = smem_best;
            o.prefetch_depth = dep;
            if (join) o.flags |= MB_LOCATE_JOIN;
            rc = time_point(o);
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != MB_OK) return rc;
    *best = bo;
    if (best_ms) *best_ms = bms;
    if (n_points) *n_points = np;
    return MB_OK;
}

extern "C" int mb_autotune(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                           const mb_opts *opts, void *stream, mb_opts *best, double *best_ms) {
    return autotune_impl(idx, seq, off, n_reads, opts, (cudaStream_t)stream, best, best_ms, nullptr, nullptr, 0,
                         nullptr);
}

extern "C" int mb_autotune_points(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                                  const mb_opts *opts, void *stream, mb_opts *best, double *best_ms, mb_opts *points,
                                  double *points_ms, uint32_t cap, uint32_t *n_points) {
    return autotune_impl(idx, seq, off, n_reads, opts, (cudaStream_t)stream, best, best_ms, points, points_ms, cap,
                         n_points);
}

// ============================================================================ second seeding round
namespace {
// window of record m: an SMEM of at least min_w bases that occurs at most max_s times
__global__ void k_win_flag(const mb_smem *__restrict__ sm, u64 nsm, u32 min_w, u32 max_s, u64 *__restrict__ flag) {
    for (u64 m = blockIdx.x * (u64)blockDim.x + threadIdx.x; m < nsm; m += (u64)gridDim.x * blockDim.x) {
        const mb_smem x = sm[m];
        flag[m] = (x.qend - x.qbeg >= min_w && x.s <= max_s && !(x.flags & MB_SMEM_OVER_MAX_OCC)) ? 1 : 0;
    }
}
// window w: read, start, length, (l' | c' << 16) with l' = floor(len / 2), c' = s + 1
__global__ void k_win_build(const mb_smem *__restrict__ sm, u64 nsm, const u64 *__restrict__ flag,
                            const u64 *__restrict__ wpos, const u8 *__restrict__ mate, uint2 *__restrict__ winfo,
                            u64 *__restrict__ wlen, u32 *__restrict__ lc, u8 *__restrict__ wmate) {
    for (u64 m = blockIdx.x * (u64)blockDim.x + threadIdx.x; m < nsm; m += (u64)gridDim.x * blockDim.x) {
        if (!flag[m]) continue;
        const mb_smem x = sm[m];
        const u64 w = wpos[m];
        const u32 len = x.qend - x.qbeg;
        winfo[w] = make_uint2(x.read, x.qbeg);
        wlen[w] = len;
        lc[w] = (len / 2) | ((u32)(x.s + 1) << 16);
        wmate[w] = mate ? mate[x.read] : 0;
    }
}
// bases of every window, one warp per window
__global__ void k_win_copy(const u8 *__restrict__ seq, const u64 *__restrict__ off, const uint2 *__restrict__ winfo,
                           const u64 *__restrict__ woff, u64 nw, u8 *__restrict__ wseq) {
    const u32 lane = threadIdx.x & 31;
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 w = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; w < nw; w += nwarps) {
        const u8 *src = seq + off[winfo[w].x] + winfo[w].y;
        const u64 b = woff[w], len = woff[w + 1] - b;
        for (u64 t = lane; t < len; t += 32) wseq[b + t] = src[t];
    }
}
// records of the windows back in read coordinates
__global__ void k_win_fix(mb_smem *__restrict__ out, u64 n, const uint2 *__restrict__ winfo) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < n; t += (u64)gridDim.x * blockDim.x) {
        const uint2 w = winfo[out[t].read];
        out[t].read = w.x;
        out[t].qbeg += w.y;
        out[t].qend += w.y;
        out[t].flags |= MB_SMEM_ROUND2;
    }
}
}  // namespace

extern "C" int mb_reseed(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                         const uint8_t *mate, const mb_smem *smem, uint64_t n_smem, const mb_opts *opts, void *stream,
                         mb_smem *out, uint64_t cap, uint64_t *n_out, uint64_t *n_hits) {
    if (!idx || !off || !n_out || (n_reads && !seq) || (n_smem && !smem)) return MB_ERR_ARG;
    *n_out = 0;
    if (n_hits) *n_hits = 0;
    if (n_reads == 0 || n_smem == 0) return MB_OK;
    u32 l, c, max_occ, flags;
    opts_defaults(opts, l, c, max_occ, flags);
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf boff, bseq, bmate, bsm;
    const void *doff = nullptr, *dseq = nullptr, *dmate = nullptr, *dsm = nullptr;
    u64 o0 = 0, o1 = 0;
    MB_CK(cudaMemcpyAsync(&o0, off, 8, cudaMemcpyDefault, st));
    MB_CK(cudaMemcpyAsync(&o1, off + n_reads, 8, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    MB_TRY(mb_stage_in(off, (size_t)(n_reads + 1) * 8, st, boff, &doff));
    if (mb_is_device_ptr(seq)) dseq = seq;
    else {
        MB_TRY(bseq.alloc(o1 - o0 + 1, st));
        MB_CK(cudaMemcpyAsync(bseq.as<u8>(), seq + o0, o1 - o0, cudaMemcpyHostToDevice, st));
        dseq = bseq.as<u8>() - o0;
    }
    if (mate) MB_TRY(mb_stage_in(mate, n_reads, st, bmate, &dmate));
    MB_TRY(mb_stage_in(smem, n_smem * sizeof(mb_smem), st, bsm, &dsm));
    // windows (Section 2.6): SMEMs of at least 2l bases occurring at most 10 times
    DevBuf bflag, bwpos, btmp, bmisc;
    MB_TRY(bflag.alloc(n_smem * 8, st));
    MB_TRY(bwpos.alloc(n_smem * 8, st));
    MB_TRY(btmp.alloc(scan_tmp_bytes(n_smem + 1), st));
    MB_TRY(bmisc.alloc(64, st));
    k_win_flag<<<grid_for(n_smem, 256), 256, 0, st>>>((const mb_smem *)dsm, n_smem, 2 * l, RESEED_MAX_OCC,
                                                      bflag.as<u64>());
    MB_KCHECK();
    MB_TRY(scan_exclusive_u64(bflag.as<u64>(), bwpos.as<u64>(), n_smem, bmisc.as<u64>(), btmp.p, st));
    u64 nw = 0;
    MB_CK(cudaMemcpyAsync(&nw, bmisc.p, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (nw == 0) return MB_OK;
    if (nw >= (1ull << 32)) return MB_ERR_ARG;
    DevBuf binfo, bwlen, blc, bwmate, bwoff, bwseq;
    MB_TRY(binfo.alloc(nw * 8, st));
    MB_TRY(bwlen.alloc(nw * 8, st));
    MB_TRY(blc.alloc(nw * 4, st));
    MB_TRY(bwmate.alloc(nw, st));
    MB_TRY(bwoff.alloc((nw + 1) * 8, st));
    k_win_build<<<grid_for(n_smem, 256), 256, 0, st>>>((const mb_smem *)dsm, n_smem, bflag.as<u64>(),
                                                       bwpos.as<u64>(), (const u8 *)dmate, binfo.as<uint2>(),
                                                       bwlen.as<u64>(), blc.as<u32>(), bwmate.as<u8>());
    MB_KCHECK();
    MB_TRY(btmp.alloc(scan_tmp_bytes(nw), st));
    MB_TRY(scan_exclusive_u64(bwlen.as<u64>(), bwoff.as<u64>(), nw, bwoff.as<u64>() + nw, btmp.p, st));
    u64 wbases = 0;
    MB_CK(cudaMemcpyAsync(&wbases, bwoff.as<u64>() + nw, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    MB_TRY(bwseq.alloc(wbases + 16, st));
    k_win_copy<<<grid_for(nw * 32, 256), 256, 0, st>>>((const u8 *)dseq, (const u64 *)doff, binfo.as<uint2>(),
                                                       bwoff.as<u64>(), nw, bwseq.as<u8>());
    MB_KCHECK();
    // the seeding pipeline on the windows, each with its own (l', c'); window bases are copied
    // unconverted, so in bisulfite mode each window is converted by its read's mate flag
    mb_opts o = opts ? *opts : mb_opts{};
    o.flags &= ~(u32)MB_COUNT;
    const u8 *wm = (flags & MB_BS3) ? bwmate.as<u8>() : nullptr;
    DevBuf bout;
    const bool out_dev = mb_is_device_ptr(out);
    u64 need = 0, nh = 0;
    int rc = mb_seed_device(idx, bwseq.as<u8>(), bwoff.as<u64>(), (u32)nw, wm, blc.as<u32>(), 0, wbases, &o, st,
                         nullptr, 0, &need, &nh);
    if (rc != MB_OK && rc != MB_ERR_CAPACITY) return rc;
    *n_out = need;
    if (need > cap) return MB_ERR_CAPACITY;
    if (need == 0) return MB_OK;
    if (!out) return MB_ERR_ARG;
    mb_smem *dout = out;
    if (!out_dev) {
        MB_TRY(bout.alloc(need * sizeof(mb_smem), st));
        dout = bout.as<mb_smem>();
    }
    MB_TRY(mb_seed_device(idx, bwseq.as<u8>(), bwoff.as<u64>(), (u32)nw, wm, blc.as<u32>(), 0, wbases, &o, st, dout,
                       need, &need, &nh));
    k_win_fix<<<grid_for(need, 256), 256, 0, st>>>(dout, need, binfo.as<uint2>());
    MB_KCHECK();
    if (!out_dev) MB_CK(cudaMemcpyAsync(out, dout, need * sizeof(mb_smem), cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    if (n_hits) *n_hits = nh;
    return MB_OK;
}
