/*
 * CPU ORACLE for the seeding stage of minibwa (arxiv 2606.15357).
 *
 * This is test infrastructure.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference leg may load it.  It shares no code,
 * header, table or constant with the CUDA library; it is slow and plain on
 * purpose, so that a reader can check it against the paper by eye.
 *
 * What it computes (paper, Section 2.1 "Definitions"):
 *   T = R . revcomp(R) . $, n = |T|, ambiguous bases of R replaced by random bases;
 *   S = suffix array of T, B[i] = T[S(i)-1] (T[-1] = $);
 *   ds-interval of P = (lo(P), lo(revcomp P), occ(P)) with lo(P) = #{i : T[i,n) < P}
 *     and occ(P) = #{i : T[i,i+|P|) = P};
 *   (l,c)-match = a substring P[i,j) with j-i >= l and occ >= c;
 *   (l,c)-SMEM  = a match contained in no other match;
 *   locate = { S(x) : k <= x < k+s } for the ds-interval (k,k',s) of an SMEM.
 * plus, as separately checked routes to the same results,
 *   pi(a,k) (Section 2.1), BackwardExt / ForwardExt (Algorithm 1),
 *   BatchFindSMEM (Algorithm 3), LocateSlow and BatchLocate (Algorithm 2),
 * and brute force by scanning T (tiny inputs only).
 *
 * Symbol coding inside the oracle: $=0, A=1, C=2, G=3, T=4 (the order of the
 * paper's alphabet with the sentinel smallest).  Read bases arrive as
 * 0..3 = A..T and 4 = N; an N never matches (occurs 0 times).
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - ambiguous reference bases: replaced by bits 63..62 of splitmix64's output
 *    function applied to (seed + (pos+1) * 0x9E3779B97F4A7C15);
 *  - a pattern containing N has ds-interval (0,0,0);
 *  - Algorithm 2's result is taken modulo n (a walk through the $ row lands on
 *    row 0, whose S value is n-1);
 *  - bisulfite mode indexes R3 = CT(R) . GA(R) (Section 2.9) in place of R.
 */
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <atomic>
#include <vector>
#include <omp.h>

typedef uint64_t u64;
typedef uint32_t u32;
typedef uint8_t u8;

namespace {

/* splitmix64 output function (Steele, Lea, Flood 2014) on a counter */
u64 mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
u8 random_base(u64 seed, u64 pos) { return (u8)(mix64(seed + (pos + 1) * 0x9E3779B97F4A7C15ULL) >> 62); }

inline u8 comp_sym(u8 a) { return a == 0 ? 0 : (u8)(5 - a); }   // $ -> $, A<->T, C<->G

struct Index {
    u64 rlen = 0;            // length of the indexed forward text (|R|, or |R3| in bisulfite mode)
    u64 n = 0;               // |T|
    std::vector<u8> T;       // T[0,n), codes 0..4
    std::vector<u32> SA;     // full suffix array
    std::vector<u8> B;       // BWT
    u64 primary = 0;         // row i with S(i) = 0 (B[i] = $)
    u64 C[5];                // C[a] = #{i : B[i] < a}
    std::vector<u32> ck;     // ck[(k/64)*5 + a] = #{i < 64*(k/64) : B[i] = a}
    u32 r = 32;              // SA sample rate
    std::vector<u32> ssa;    // ssa[x] = S(x*r)
};

/* ---------------------------------------------------------------- suffix array, BWT */

/* Suffix order by direct comparison of the two suffixes (T ends with the unique $). */
struct SuffixLess {
    const u8 *T; u64 off;
    bool operator()(u32 a, u32 b) const {
        u64 q = off;
        while (T[a + q] == T[b + q]) ++q;
        return T[a + q] < T[b + q];
    }
};

/*
 * S by sorting all suffixes: a counting pass on the first K symbols (base 5,
 * positions past the end read as 0) puts them into buckets in order, then each
 * bucket is sorted with the plain suffix comparison.
 */
void build_sa(Index &X, int threads) {
    const u64 n = X.n;
    const u8 *T = X.T.data();
    int K = 1;
    u64 nb = 5;
    while (K < 11 && nb * 5 <= std::max<u64>(n, 25)) { ++K; nb *= 5; }
    auto key = [&](u64 i) {
        u64 v = 0;
        for (int q = 0; q < K; ++q) v = v * 5 + (i + q < n ? T[i + q] : 0);
        return v;
    };
    std::vector<std::atomic<u32>> cnt(nb + 1);
    for (auto &c : cnt) c.store(0, std::memory_order_relaxed);
#pragma omp parallel for num_threads(threads) schedule(static)
    for (u64 i = 0; i < n; ++i) cnt[key(i) + 1].fetch_add(1, std::memory_order_relaxed);
    std::vector<u64> start(nb + 1, 0);
    for (u64 b = 0; b < nb; ++b) start[b + 1] = start[b] + cnt[b + 1].load(std::memory_order_relaxed);
    for (u64 b = 0; b <= nb; ++b) cnt[b].store(0, std::memory_order_relaxed);
    X.SA.assign(n, 0);
    u32 *SA = X.SA.data();
#pragma omp parallel for num_threads(threads) schedule(static)
    for (u64 i = 0; i < n; ++i) {
        u64 b = key(i);
        SA[start[b] + cnt[b].fetch_add(1, std::memory_order_relaxed)] = (u32)i;
    }
    SuffixLess less{T, (u64)K};
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4096)
    for (u64 b = 0; b < nb; ++b)
        if (start[b + 1] - start[b] > 1) std::sort(SA + start[b], SA + start[b + 1], less);
}

void build_index(Index &X, const u8 *ref, u64 len, u64 seed, int bs3, u32 r, int threads) {
    /* R: ambiguous bases -> random bases */
    std::vector<u8> R(len);
    for (u64 i = 0; i < len; ++i) R[i] = ref[i] < 4 ? ref[i] : random_base(seed, i);
    if (bs3) {   /* R3 = CT(R) . GA(R) */
        std::vector<u8> R3(2 * len);
        for (u64 i = 0; i < len; ++i) {
            R3[i] = R[i] == 1 ? 3 : R[i];            // C -> T
            R3[len + i] = R[i] == 2 ? 0 : R[i];      // G -> A
        }
        R.swap(R3);
    }
    const u64 m = R.size();
    X.rlen = m;
    X.n = 2 * m + 1;
    X.T.assign(X.n + 1, 0);
    for (u64 i = 0; i < m; ++i) {
        X.T[i] = (u8)(R[i] + 1);
        X.T[m + i] = comp_sym((u8)(R[m - 1 - i] + 1));
    }
    X.T[X.n - 1] = 0;   // $
    X.T[X.n] = 0;       // guard, outside T
    build_sa(X, threads);
    /* B[i] = T[S(i) - 1] with T[-1] = $ */
    X.B.resize(X.n);
    for (u64 i = 0; i < X.n; ++i) {
        u64 p = X.SA[i];
        X.B[i] = p == 0 ? 0 : X.T[p - 1];
        if (p == 0) X.primary = i;
    }
    u64 tot[5] = {0, 0, 0, 0, 0};
    X.ck.assign((X.n / 64 + 1) * 5, 0);
    for (u64 i = 0; i < X.n; ++i) {
        if (i % 64 == 0) for (int a = 0; a < 5; ++a) X.ck[(i / 64) * 5 + a] = (u32)tot[a];
        ++tot[X.B[i]];
    }
    if (X.n % 64 == 0) for (int a = 0; a < 5; ++a) X.ck[(X.n / 64) * 5 + a] = (u32)tot[a];
    u64 acc = 0;
    for (int a = 0; a < 5; ++a) { X.C[a] = acc; acc += tot[a]; }
    X.r = r;
    X.ssa.resize((X.n + r - 1) / r);
    for (u64 x = 0; x < X.n; x += r) X.ssa[x / r] = X.SA[x];
}

/* ---------------------------------------------------------------- pi and Algorithm 1 */

/* #{i < k : B[i] = a} */
u64 occ(const Index &X, u8 a, u64 k) {
    u64 c = X.ck[(k / 64) * 5 + a];
    for (u64 i = (k / 64) * 64; i < k; ++i) c += X.B[i] == a;
    return c;
}
/* pi(a,k) = #{i : B[i] < a} + #{i < k : B[i] = a} */
u64 pi(const Index &X, u8 a, u64 k) { return X.C[a] + occ(X, a, k); }

struct DS { u64 k, kr, s; };

/* Algorithm 1, BackwardExt: ds-interval of aP from that of P.  a in 1..4; a = 5 is N. */
DS backward_ext(const Index &X, DS v, u8 a) {
    if (a > 4) return DS{0, 0, 0};
    u8 ac = comp_sym(a);
    for (u8 b = 0; b < ac; ++b) {   // every b < complement(a), b may be $
        u8 bc = comp_sym(b);
        v.kr += pi(X, bc, v.k + v.s) - pi(X, bc, v.k);
    }
    u64 lo = pi(X, a, v.k), hi = pi(X, a, v.k + v.s);
    return DS{lo, v.kr, hi - lo};
}
/* Algorithm 1, ForwardExt: ds-interval of Pa */
DS forward_ext(const Index &X, DS v, u8 a) {
    if (a > 4) return DS{0, 0, 0};
    DS w = backward_ext(X, DS{v.kr, v.k, v.s}, comp_sym(a));
    return DS{w.kr, w.k, w.s};
}

/* ---------------------------------------------------------------- definitions by the SA */

/* compare suffix T[p,n) with pattern P[0,m): <0, 0 (P is a prefix of the suffix), >0 */
int cmp_suffix(const Index &X, u64 p, const u8 *P, u64 m) {
    for (u64 q = 0; q < m; ++q) {
        u8 t = X.T[p + q];
        if (t != P[q]) return t < P[q] ? -1 : 1;   // $ (0) ends the suffix and is smallest
    }
    return 0;
}
/* lo(P) = #{i : T[i,n) < P}; hi(P) = lo(P) + occ(P).  P in codes 1..4 */
void sa_range(const Index &X, const u8 *P, u64 m, u64 *lo, u64 *hi) {
    u64 a = 0, b = X.n;
    while (a < b) { u64 x = (a + b) / 2; if (cmp_suffix(X, X.SA[x], P, m) < 0) a = x + 1; else b = x; }
    *lo = a;
    b = X.n;
    while (a < b) { u64 x = (a + b) / 2; if (cmp_suffix(X, X.SA[x], P, m) <= 0) a = x + 1; else b = x; }
    *hi = a;
}
/* ds-interval by definition; P in read codes (0..3, 4 = N) */
DS ds_def(const Index &X, const u8 *P, u64 m) {
    std::vector<u8> f(m), rc(m);
    for (u64 q = 0; q < m; ++q) {
        if (P[q] > 3) return DS{0, 0, 0};
        f[q] = (u8)(P[q] + 1);
        rc[m - 1 - q] = comp_sym(f[q]);
    }
    u64 lo, hi, lor, hir;
    sa_range(X, f.data(), m, &lo, &hi);
    sa_range(X, rc.data(), m, &lor, &hir);
    return DS{lo, lor, hi - lo};
}

struct Smem { u32 read, qbeg, qend, pad; u64 k, kr, s; };

/*
 * (l,c)-SMEMs of one read by the definition.  For every start i let r(i) be
 * the largest j with occ(P[i,j)) >= c (r(i) = i if no base matches).  occ
 * never grows when a match is extended, so the matches starting at i are the
 * P[i,j) with i+l <= j <= r(i), and r is non-decreasing in i.  A match is
 * contained in another one iff it can be extended by one base on the left or
 * on the right and stay a match.  Hence the SMEMs are exactly the [i, r(i))
 * with r(i) - i >= l and (i = 0 or r(i-1) < r(i)).
 * r(i) is found by narrowing the SA range of P[i, .) one symbol at a time.
 */
void smem_def_read(const Index &X, const u8 *P, u32 m, u32 rid, u32 l, u32 c, std::vector<Smem> &out) {
    std::vector<u8> f(m);
    for (u32 q = 0; q < m; ++q) f[q] = P[q] < 4 ? (u8)(P[q] + 1) : 5;
    u64 rprev = 0;
    for (u32 i = 0; i < m; ++i) {
        u64 j = std::max<u64>(i, rprev);
        u64 lo = 0, hi = X.n;
        if (j > i) sa_range(X, f.data() + i, j - i, &lo, &hi);
        while (j < m && f[j] <= 4) {
            /* sub-range of [lo,hi) whose suffixes continue with f[j] at offset j-i */
            u64 d = j - i, a = lo, b = hi;
            while (a < b) { u64 x = (a + b) / 2; if (X.T[X.SA[x] + d] < f[j]) a = x + 1; else b = x; }
            u64 nlo = a;
            b = hi;
            while (a < b) { u64 x = (a + b) / 2; if (X.T[X.SA[x] + d] <= f[j]) a = x + 1; else b = x; }
            u64 nhi = a;
            if (nhi - nlo < c) break;
            lo = nlo; hi = nhi; ++j;
        }
        if (j - i >= l && (i == 0 || rprev < j)) {
            DS v = ds_def(X, P + i, j - i);
            out.push_back(Smem{rid, i, (u32)j, 0, v.k, v.kr, v.s});
        }
        rprev = j;
    }
}

/* Work of Algorithm 1 calls, for the measurement's algorithmic bytes: one step per call with a
 * base (an N reads nothing); the occurrence values a call needs sit at rows p and p+s of the
 * strand it extends (p = k backwards, k' forwards), i.e. in one block of `block_rows` rows when
 * both rows fall in it, else in two. */
struct Work { u64 steps = 0, blocks = 0, lookups = 0; u64 block_rows = 64; };
void count_ext(Work *w, u64 p, u64 s, u8 a) {
    if (!w || a > 4) return;
    w->steps += 1;
    w->blocks += (p / w->block_rows == (p + s) / w->block_rows) ? 1 : 2;
}

/*
 * Algorithm 3 (Section 2.5) for one read P of m bases (oracle codes, 5 = N).  Algorithm 3 keeps
 * one queue entry per read at any time, so a read's extensions happen in a fixed order whatever
 * the other reads do; the batch, the queue and the prefetching only change when they happen.
 * Here each read runs alone, start to end, as three nested scans over the start i of the next
 * candidate match:
 *   - check that the window P[i, i+l) occurs at least c times by extending backwards from its
 *     last base; at a failing base t no window starting at or before t can match, so the scan
 *     moves on to i = t + 1 (or the read ends when that window would pass the end of P);
 *   - extend the match forwards as long as it occurs at least c times and report it as an SMEM
 *     with the ds-interval of its last successful extension;
 *   - from the base e where the forward extension failed, extend backwards over P[e], P[e-1], ...
 *     down to just above i; the base t where this fails (or i itself) bounds the next start:
 *     every match holding P[e] starts after t, and the scan goes back to the window check at
 *     t + 1.
 * The extensions are BackwardExt / ForwardExt of Algorithm 1, in the order Algorithm 3 makes
 * them for this read, so the work counts are Algorithm 3's.
 *
 * With K > 0, the ds-interval cache of Section 2.5 (the intervals of all K-mers) stands in for the
 * first K backward extensions from the whole interval, read as follows: the cached value of the
 * K-mer P[t-K+1, t] is its ds-interval by definition (what K BackwardExt steps from the whole
 * interval give).  In the window check it is used when the K-mer lies inside the window and holds
 * no N; if the K-mer occurs fewer than c times, no window starting at or before its first base x
 * can match and the scan moves on to x + 1.  Looking for the next start it is used once, when the
 * K-mer lies above i and holds no N; if it fails there the extensions go one base at a time (the
 * exact failing base is needed).  The SMEMs are the same with or without it.
 */
static bool has_n(const u8 *P, int64_t a, int64_t b) {
    for (int64_t q = a; q < b; ++q)
        if (P[q] > 4) return true;
    return false;
}
static DS kmer_ds(const Index &X, const u8 *P, int64_t a, u32 K) {   /* P in oracle codes 1..4 */
    std::vector<u8> r(K);
    for (u32 q = 0; q < K; ++q) r[q] = (u8)(P[a + q] - 1);
    return ds_def(X, r.data(), K);
}
void smem_alg3_read(const Index &X, const u8 *P, int64_t m, u32 rid, u32 l, u32 c, std::vector<Smem> &out,
                    Work *work, u32 K = 0) {
    const DS whole{0, 0, X.n};
    const int64_t L = (int64_t)l;
    if (L - 1 >= m) return;                       // the read is shorter than l
    int64_t i = 0;
    for (;;) {
        /* window check of P[i, i+l) */
        DS v = whole;
        int64_t t = i + L - 1;
        if (K && L >= (int64_t)K && !has_n(P, t - K + 1, t + 1)) {
            if (work) work->lookups += 1;
            const DS w = kmer_ds(X, P, t - K + 1, K);
            if (w.s < c) {                        // no window starting at or before x = t-K+1
                const int64_t x = t - K + 1;
                if (x + L < m) { i = x + 1; continue; }
                return;
            }
            v = w;
            t -= K;
        }
        for (; t >= i; --t) {
            count_ext(work, v.k, v.s, P[t]);
            const DS w = backward_ext(X, v, P[t]);
            if (w.s < c) break;
            v = w;
        }
        if (t >= i) {                             // failed at base t
            if (t + L < m) { i = t + 1; continue; }
            return;
        }
        /* forward extension of the match P[i, e) */
        int64_t e = i + L;
        while (e < m) {
            count_ext(work, v.kr, v.s, P[e]);
            const DS w = forward_ext(X, v, P[e]);
            if (w.s < c) break;
            v = w;
            ++e;
        }
        out.push_back(Smem{rid, (u32)i, (u32)e, 0, v.k, v.kr, v.s});
        if (e == m) return;
        /* the next start: backwards from the failing base e, not below i + 1 */
        v = whole;
        t = e;
        if (K && t - (int64_t)K + 1 > i && !has_n(P, t - K + 1, t + 1)) {
            if (work) work->lookups += 1;
            const DS w = kmer_ds(X, P, t - K + 1, K);
            if (w.s >= c) {
                v = w;
                t -= K;
            }
        }
        for (; t > i; --t) {
            count_ext(work, v.k, v.s, P[t]);
            const DS w = backward_ext(X, v, P[t]);
            if (w.s < c) break;
            v = w;
        }
        if (t > i && t + L >= m) return;          // failed at t, and no window fits after it
        i = t + 1;
    }
}

/* Algorithm 3 over a batch: every read on its own (see smem_alg3_read), reads in parallel. */
void smem_alg3(const Index &X, const u8 *seq, const u64 *off, u32 nr, u32 l, u32 c,
               std::vector<std::vector<Smem>> &out, Work *work = nullptr, int threads = 0, u32 K = 0) {
    u64 steps = 0, blocks = 0, lookups = 0;
    const u64 br = work ? work->block_rows : 64;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 16) \
    reduction(+ : steps, blocks, lookups)
    for (u32 rd = 0; rd < nr; ++rd) {
        const int64_t m = (int64_t)(off[rd + 1] - off[rd]);
        std::vector<u8> P(m);
        for (int64_t q = 0; q < m; ++q) P[q] = seq[off[rd] + q] < 4 ? (u8)(seq[off[rd] + q] + 1) : 5;
        Work w;
        w.block_rows = br;
        smem_alg3_read(X, P.data(), m, rd, l, c, out[rd], work ? &w : nullptr, K);
        steps += w.steps;
        blocks += w.blocks;
        lookups += w.lookups;
    }
    if (work) {
        work->steps += steps;
        work->blocks += blocks;
        work->lookups += lookups;
    }
}

/* ---------------------------------------------------------------- Algorithm 2 */

/* LocateSlow: LF-walk each row to a sampled row; result taken modulo n */
u64 locate_slow_one(const Index &X, u64 k) {
    u64 i = 0;
    while (k % X.r != 0) { k = pi(X, X.B[k], k); ++i; }
    return (i + X.ssa[k / X.r]) % X.n;
}

/* Work of one LocateSlow walk under the reading that the $ row counts as sampled with S = 0
 * (the walk stops there): LF steps taken, and whether it ends by reading a sampled S value. */
void locate_work(const Index &X, u64 k, u64 &steps, u64 &sa_reads) {
    while (k % X.r != 0 && k != X.primary) { k = pi(X, X.B[k], k); ++steps; }
    if (k % X.r == 0) ++sa_reads;
}

/* BatchLocate: the same walks, advanced level by level over the set E */
void batch_locate(const Index &X, const u64 *rows, u64 m, u64 *pos) {
    struct W { u64 k, idx; };
    std::vector<W> E(m), E2;
    for (u64 q = 0; q < m; ++q) E[q] = W{rows[q], q};
    u64 i = 0;
    while (!E.empty()) {
        E2.clear();
        for (const W &w : E) {
            if (w.k % X.r == 0) pos[w.idx] = (i + X.ssa[w.k / X.r]) % X.n;
            else E2.push_back(W{pi(X, X.B[w.k], w.k), w.idx});
        }
        ++i;
        E.swap(E2);
    }
}

/* ---------------------------------------------------------------- brute force (tiny T) */

/*
 * SMEMs of one read by scanning T: cnt[i][m] = #{t : T[t,t+m) = P[i,i+m)} from
 * the match length of every (t, i) pair; lo() by comparing every suffix.
 */
u64 lo_scan(const u8 *T, u64 n, const u8 *P, u64 m) {
    u64 c = 0;
    for (u64 t = 0; t < n; ++t) {
        u64 q = 0;
        while (q < m && T[t + q] == P[q]) ++q;
        if (q < m && T[t + q] < P[q]) ++c;    // T[t,n) < P
    }
    return c;
}

void smem_brute_read(const u8 *T, u64 n, const u8 *Pin, u32 m, u32 rid, u32 l, u32 c, std::vector<Smem> &out) {
    std::vector<u8> P(m);
    for (u32 q = 0; q < m; ++q) P[q] = Pin[q] < 4 ? (u8)(Pin[q] + 1) : 7;  // N matches nothing
    std::vector<u64> cnt((size_t)m * (m + 2), 0);   // cnt[i*(m+2) + len]
    std::vector<u32> row(m + 1, 0), nrow(m + 1, 0);  // match length of (t, i), rolling over t
    for (int64_t t = (int64_t)n - 1; t >= 0; --t) {
        for (u32 i = 0; i < m; ++i) nrow[i] = T[t] == P[i] ? 1 + row[i + 1] : 0;
        nrow[m] = 0;
        for (u32 i = 0; i < m; ++i) ++cnt[(size_t)i * (m + 2) + nrow[i]];
        row.swap(nrow);
    }
    /* occ(P[i,i+len)) = #{t : matchlen(t,i) >= len} */
    for (u32 i = 0; i < m; ++i)
        for (int64_t L = m; L >= 0; --L) cnt[(size_t)i * (m + 2) + L] += cnt[(size_t)i * (m + 2) + L + 1];
    auto occ_of = [&](int64_t i, int64_t j) -> u64 { return cnt[(size_t)i * (m + 2) + (j - i)]; };
    auto is_match = [&](int64_t i, int64_t j) -> bool {
        return i >= 0 && j <= (int64_t)m && j - i >= (int64_t)l && occ_of(i, j) >= c;
    };
    for (int64_t i = 0; i < (int64_t)m; ++i)
        for (int64_t j = i + l; j <= (int64_t)m; ++j) {
            if (!is_match(i, j)) continue;
            if (is_match(i - 1, j) || is_match(i, j + 1)) continue;   // contained in a longer match
            std::vector<u8> rc(j - i);
            for (int64_t q = i; q < j; ++q) rc[j - 1 - q] = comp_sym(P[q]);
            out.push_back(Smem{rid, (u32)i, (u32)j, 0, lo_scan(T, n, P.data() + i, j - i),
                               lo_scan(T, n, rc.data(), j - i), occ_of(i, j)});
        }
}

struct Result { std::vector<Smem> smem; std::vector<u64> u64s; };

}  // namespace

/* ================================================================ C interface for the tests */
extern "C" {

void *orc_index_build(const u8 *ref, u64 len, u64 seed, int bs3, u32 sa_rate, int threads) {
    Index *X = new Index;
    build_index(*X, ref, len, seed, bs3, sa_rate, threads > 0 ? threads : omp_get_max_threads());
    return X;
}
void orc_index_free(void *x) { delete (Index *)x; }
u64 orc_n(void *x) { return ((Index *)x)->n; }
u64 orc_rlen(void *x) { return ((Index *)x)->rlen; }
u64 orc_primary(void *x) { return ((Index *)x)->primary; }
void orc_C(void *x, u64 *out) { memcpy(out, ((Index *)x)->C, sizeof(u64) * 5); }
void orc_text(void *x, u8 *out) { memcpy(out, ((Index *)x)->T.data(), ((Index *)x)->n); }
void orc_sa(void *x, u32 *out) { memcpy(out, ((Index *)x)->SA.data(), ((Index *)x)->n * 4); }
void orc_bwt(void *x, u8 *out) { memcpy(out, ((Index *)x)->B.data(), ((Index *)x)->n); }
void orc_ssa(void *x, u32 *out) { memcpy(out, ((Index *)x)->ssa.data(), ((Index *)x)->ssa.size() * 4); }
u64 orc_pi(void *x, u8 a, u64 k) { return pi(*(Index *)x, a, k); }

void orc_ds_def(void *x, const u8 *P, u64 m, u64 *out) {
    DS v = ds_def(*(Index *)x, P, m);
    out[0] = v.k; out[1] = v.kr; out[2] = v.s;
}
/* ds-interval by definition of npat patterns of length m each (row-major), out = 3 u64 each */
void orc_ds_def_batch(void *x, const u8 *pats, u64 npat, u64 m, u64 *out, int threads) {
    const Index &X = *(Index *)x;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(static)
    for (u64 q = 0; q < npat; ++q) {
        DS v = ds_def(X, pats + q * m, m);
        out[3 * q] = v.k; out[3 * q + 1] = v.kr; out[3 * q + 2] = v.s;
    }
}
/* a in read codes (0..3 = A..T, 4 = N) */
void orc_backward_ext(void *x, const u64 *in, u8 a, u64 *out) {
    DS v = backward_ext(*(Index *)x, DS{in[0], in[1], in[2]}, a < 4 ? (u8)(a + 1) : 5);
    out[0] = v.k; out[1] = v.kr; out[2] = v.s;
}
void orc_forward_ext(void *x, const u64 *in, u8 a, u64 *out) {
    DS v = forward_ext(*(Index *)x, DS{in[0], in[1], in[2]}, a < 4 ? (u8)(a + 1) : 5);
    out[0] = v.k; out[1] = v.kr; out[2] = v.s;
}

/* method: 0 = definition, 1 = Algorithm 3.  Returns a result handle; records are per read in
 * read order, ascending qbeg within a read. */
void *orc_smem(void *x, const u8 *seq, const u64 *off, u32 nr, u32 l, u32 c, int method, int threads) {
    const Index &X = *(Index *)x;
    Result *res = new Result;
    std::vector<std::vector<Smem>> per(nr);
    if (method == 1 || method == 2) {   /* 2: with the 10-mer cache of Section 2.5 */
        Work w;
        smem_alg3(X, seq, off, nr, l, c, per, method == 2 ? &w : nullptr, threads, method == 2 ? 10u : 0u);
        for (auto &v : per) std::sort(v.begin(), v.end(), [](const Smem &a, const Smem &b) { return a.qbeg < b.qbeg; });
    } else {
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 16)
        for (u32 rd = 0; rd < nr; ++rd)
            smem_def_read(X, seq + off[rd], (u32)(off[rd + 1] - off[rd]), rd, l, c, per[rd]);
    }
    for (auto &v : per) res->smem.insert(res->smem.end(), v.begin(), v.end());
    return res;
}

/* brute force over the text T (oracle coding, length n, T[n-1] = $) */
void *orc_smem_brute(const u8 *T, u64 n, const u8 *seq, const u64 *off, u32 nr, u32 l, u32 c, int threads) {
    Result *res = new Result;
    std::vector<u8> Tg(T, T + n);
    Tg.resize(n + 1, 0);
    std::vector<std::vector<Smem>> per(nr);
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 1)
    for (u32 rd = 0; rd < nr; ++rd)
        smem_brute_read(Tg.data(), n, seq + off[rd], (u32)(off[rd + 1] - off[rd]), rd, l, c, per[rd]);
    for (auto &v : per) res->smem.insert(res->smem.end(), v.begin(), v.end());
    return res;
}

u64 orc_result_nsmem(void *r) { return ((Result *)r)->smem.size(); }
/* copies records as 6 u64 each: read, qbeg, qend, k, kr, s */
void orc_result_smem(void *r, u64 *out) {
    const auto &v = ((Result *)r)->smem;
    for (size_t q = 0; q < v.size(); ++q) {
        out[6 * q + 0] = v[q].read; out[6 * q + 1] = v[q].qbeg; out[6 * q + 2] = v[q].qend;
        out[6 * q + 3] = v[q].k; out[6 * q + 4] = v[q].kr; out[6 * q + 5] = v[q].s;
    }
}
void orc_result_free(void *r) { delete (Result *)r; }

/* locate by the definition: pos[q] = S(rows[q]) */
void orc_locate_sa(void *x, const u64 *rows, u64 m, u64 *pos, int threads) {
    const Index &X = *(Index *)x;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(static)
    for (u64 q = 0; q < m; ++q) pos[q] = X.SA[rows[q]];
}
/* Algorithm 2, LocateSlow */
void orc_locate_slow(void *x, const u64 *rows, u64 m, u64 *pos, int threads) {
    const Index &X = *(Index *)x;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 64)
    for (u64 q = 0; q < m; ++q) pos[q] = locate_slow_one(X, rows[q]);
}
/* Algorithm 2, BatchLocate (single thread, one set E) */
void orc_batch_locate(void *x, const u64 *rows, u64 m, u64 *pos) { batch_locate(*(Index *)x, rows, m, pos); }

/* Work counts for the algorithmic bytes: Algorithm 3 over the reads, with the K-mer cache when
 * K > 0 (out: extension steps, blocks of `block_rows` rows read, cache lookups), and Algorithm 2
 * over the rows (out: LF steps, S reads). */
void orc_count_alg3(void *x, const u8 *seq, const u64 *off, u32 nr, u32 l, u32 c, u64 block_rows, u32 K,
                    u64 *out) {
    std::vector<std::vector<Smem>> per(nr);
    Work w;
    w.block_rows = block_rows;
    smem_alg3(*(Index *)x, seq, off, nr, l, c, per, &w, 0, K);
    out[0] = w.steps;
    out[1] = w.blocks;
    out[2] = w.lookups;
}
void orc_count_locate(void *x, const u64 *rows, u64 m, u64 *out, int threads) {
    const Index &X = *(Index *)x;
    u64 steps = 0, sa = 0;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 64) \
    reduction(+ : steps, sa)
    for (u64 q = 0; q < m; ++q) locate_work(X, rows[q], steps, sa);
    out[0] = steps;
    out[1] = sa;
}

/* Work of locate with walks that join, over the sorted distinct rows R, in 2^bits passes: row y
 * belongs to pass (y * 2654435761 mod 2^32) >> (32 - bits) (Knuth's multiplicative hash).  From
 * each row, LF steps until a sampled row or the $ row (an S read for a sampled row), or, after at
 * least one step, a row of R of an earlier pass than the walk's own (the walk takes that row's
 * position plus its distance).  out: LF steps, S reads, walks that stopped at a row of R. */
void orc_count_locate_join(void *x, const u64 *rows, u64 m, u32 bits, u64 *out, int threads) {
    const Index &X = *(Index *)x;
    std::vector<u64> R(rows, rows + m);
    std::sort(R.begin(), R.end());
    auto pass = [bits](u64 y) -> u32 {
        return bits == 0 ? 0u : (u32)(((u32)y * 2654435761u) >> (32 - bits));
    };
    u64 steps = 0, sa = 0, links = 0;
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 64) \
    reduction(+ : steps, sa, links)
    for (u64 q = 0; q < m; ++q) {
        u64 k = rows[q], t = 0;
        const u32 own = pass(rows[q]);
        for (;;) {
            if (k % X.r == 0) { ++sa; break; }
            if (k == X.primary) break;
            if (t > 0 && pass(k) < own && std::binary_search(R.begin(), R.end(), k)) { ++links; break; }
            k = pi(X, X.B[k], k);
            ++t;
        }
        steps += t;
    }
    out[0] = steps;
    out[1] = sa;
    out[2] = links;
}

}  // extern "C"
