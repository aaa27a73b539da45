/*
 * CPU comparator of the seeding stage: the paper's own CPU design (Sections 2.3-2.5), built to be
 * timed next to the GPU path as context.  It is not the oracle and not part of the product path
 * (the library never calls it); bench.py times it on the host cores.
 *
 *  - Occurrence blocks as the paper lays them out for a 64-byte cache line (Section 2.2): per
 *    128 BWT rows, the counts of A, C, G, T before the block (4 x u64) and the 128 symbols at 2
 *    bits (4 x u64).  The $ row is stored as A and left out of the counts.
 *  - Algorithm 3 over a batch of reads that take turns, one memory access per read per turn;
 *    after its turn a read prefetches the blocks holding the two rows its next extension reads
 *    (the prefetching of Section 2.5), so that by its next turn the data is in cache.
 *  - The ds-intervals of all 10-mers precomputed (Section 2.5); a stage-1 entry that starts from
 *    the empty interval takes the 10 backward steps as one table lookup.  A failing 10-mer
 *    restarts stage 1 at its second base; stage 3 tries the table once and steps otherwise.
 *  - BatchLocate (Algorithm 2) over the rows of every kept SMEM of the batch, level by level,
 *    prefetching the block of each next row.
 * OpenMP over batches of reads.
 */
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <vector>
#include <omp.h>

typedef uint64_t u64;
typedef uint32_t u32;
typedef uint8_t u8;

namespace {

struct Block {
    u64 cnt[4];   // A, C, G, T in B[0, 128 b), $ excluded
    u64 w[4];     // row q of the block at bits 2 (q % 32) of w[q / 32]; $ as A
};

struct Index {
    u64 n = 0, primary = 0;
    u64 C[4] = {0, 0, 0, 0};   // #{B[i] < a} for a = A, C, G, T ($ counted)
    std::vector<Block> blk;
    std::vector<u32> ssa;       // S(x r)
    u32 r = 32;
    std::vector<u64> kmer;      // 4^10 x (k, k', s)
};

constexpr u32 KTAB = 10;
constexpr u64 M55 = 0x5555555555555555ULL;

inline const Block &block_of(const Index &X, u64 x) { return X.blk[x >> 7]; }
inline void prefetch_row(const Index &X, u64 x) { __builtin_prefetch(&X.blk[x >> 7], 0, 0); }

// #{rows before m in word w (32 rows) holding code a}, m in 0..32
inline u32 count_word(u64 w, u32 a, u32 m) {
    if (m == 0) return 0;
    const u64 y = ~(w ^ (M55 * a));                 // 11 in every 2-bit field equal to a
    u64 eq = y & (y >> 1) & M55;
    if (m < 32) eq &= (1ULL << (2 * m)) - 1;
    return (u32)__builtin_popcountll(eq);
}
// #{rows before m in word w holding a code <= a}
inline u32 count_le_word(u64 w, u32 a, u32 m) {
    u32 c = 0;
    for (u32 b = 0; b <= a; ++b) c += count_word(w, b, m);
    return c;
}

// occurrences of code a (and of codes <= a) in B[0, x), $ excluded
inline void occ2(const Index &X, u64 x, u32 a, u64 &na, u64 &nle) {
    const Block &B = block_of(X, x);
    const u32 m = (u32)(x & 127);
    na = B.cnt[a];
    nle = 0;
    for (u32 b = 0; b <= a; ++b) nle += B.cnt[b];
    for (u32 q = 0; q < 4; ++q) {
        const int take = (int)m - 32 * (int)q;
        if (take <= 0) break;
        const u32 t = take > 32 ? 32u : (u32)take;
        na += count_word(B.w[q], a, t);
        nle += count_le_word(B.w[q], a, t);
    }
    if (X.primary < x && (X.primary >> 7) == (x >> 7)) {   // the $ row counted as A above
        if (a == 0) na -= 1;
        nle -= 1;
    }
}

struct DS { u64 k, kr, s; };

// Algorithm 1: BackwardExt by base a (0..3); a > 3 (N) gives the empty interval
inline DS backward_ext(const Index &X, DS v, u32 a) {
    if (a > 3) return DS{0, 0, 0};
    u64 na0, nle0, na1, nle1;
    occ2(X, v.k, a, na0, nle0);
    occ2(X, v.k + v.s, a, na1, nle1);
    return DS{X.C[a] + na0, v.kr + v.s - (nle1 - nle0), na1 - na0};
}
inline DS forward_ext(const Index &X, DS v, u32 a) {
    if (a > 3) return DS{0, 0, 0};
    const DS w = backward_ext(X, DS{v.kr, v.k, v.s}, 3 - a);
    return DS{w.kr, w.k, w.s};
}

inline u64 lf(const Index &X, u64 x) {   // x is not the $ row
    const Block &B = block_of(X, x);
    const u32 m = (u32)(x & 127);
    const u32 a = (u32)((B.w[m >> 5] >> (2 * (m & 31))) & 3);
    u64 na, nle;
    occ2(X, x, a, na, nle);
    return X.C[a] + na;
}

struct Rec { u32 read, qbeg, qend; u64 k, kr, s; };

// Where one read stands in Algorithm 3: stage u (1: checking the window P[i, j] backwards from
// j, 2: extending P[i, j) forwards, 3: looking backwards from j for the next start), the bounds
// and the ds-interval so far.  `tried`: stage 3 already consulted the 10-mer table.
struct Cursor {
    u32 rd;
    u8 u, tried;
    int i, j;
    DS v;
};

// Moves read e through Algorithm 3 up to and including its next memory access (one extension,
// or one table lookup plus at most one extension) and reports it; returns false when the read
// has no work left.  SMEMs found on the way go to `out`.
//
// The 10-mer table (Section 2.5) replaces the first 10 backward steps from the empty interval.
// A failing 10-mer in stage 1 restarts the window at its second base (no window starting at or
// before its first base can match); stage 3 needs the exact failing base, so it tries the table
// once and steps otherwise.
bool advance(const Index &X, const u8 *P, int L, u32 l, u32 c, Cursor &e, std::vector<Rec> &out) {
    const DS whole{0, 0, X.n};
    const int K = (int)KTAB;
    auto restart = [&](int x) {   // stage 1 at the window starting at x
        e.u = 1;
        e.tried = 0;
        e.i = x;
        e.j = x + (int)l - 1;
        e.v = whole;
    };
    for (;;) {
        if (e.u == 1 && e.j < e.i) {            // the window matches: extend it forwards
            e.u = 2;
            e.j = e.i + (int)l;
            continue;
        }
        if (e.u == 3 && e.j <= e.i) {           // every base down to i + 1 extends: next start i + 1
            restart(e.i + 1);
            continue;
        }
        if (e.u == 2) {
            if (e.j == L) {                     // the match reaches the end of the read
                out.push_back(Rec{e.rd, (u32)e.i, (u32)e.j, e.v.k, e.v.kr, e.v.s});
                return false;
            }
            const DS w = forward_ext(X, e.v, P[e.j]);
            if (w.s >= c) {
                e.v = w;
                ++e.j;
            } else {                            // the SMEM is P[i, j); look back from P[j]
                out.push_back(Rec{e.rd, (u32)e.i, (u32)e.j, e.v.k, e.v.kr, e.v.s});
                e.u = 3;
                e.tried = 0;
                e.v = whole;
            }
            return true;
        }
        // stages 1 and 3: one backward extension by P[j], the first K of them from the table
        const bool fits = e.u == 1 ? e.j - K + 1 >= e.i : e.j - K + 1 > e.i;
        if (e.v.s == X.n && l >= KTAB && fits && (e.u == 1 || !e.tried)) {
            u32 code = 0;
            bool ok = true;
            for (int t = 0; t < K && ok; ++t) {
                const u32 b = P[e.j - K + 1 + t];
                ok = b <= 3;
                code |= (b & 3u) << (2 * t);
            }
            if (ok) {
                const u64 *t = &X.kmer[3 * (u64)code];
                if (t[2] >= c) {
                    e.v = DS{t[0], t[1], t[2]};
                    e.j -= K;
                    return true;
                }
                if (e.u == 1) {
                    const int x = e.j - K + 1;
                    if (x + (int)l >= L) return false;
                    restart(x + 1);
                    return true;
                }
                e.tried = 1;
            }
        }
        const DS w = backward_ext(X, e.v, P[e.j]);
        if (w.s >= c) {
            e.v = w;
            --e.j;
            return true;
        }
        if (e.j + (int)l >= L) return false;    // no window fits after the failing base
        restart(e.j + 1);
        return true;
    }
}

// Algorithm 3 over reads [r0, r1), batched as in Section 2.5: the reads take turns, one memory
// access each per turn, and after its turn a read prefetches the blocks its next extension reads
// (rows k and k+s backwards, k' and k'+s forwards), so that the data is in cache by its next turn
// while the other reads work.  Records per read in ascending qbeg.
void batch_find_smem(const Index &X, const u8 *seq, const u64 *off, u32 r0, u32 r1, u32 l, u32 c,
                     std::vector<Rec> &out) {
    std::vector<std::vector<Rec>> per(r1 - r0);
    std::vector<Cursor> turn;
    turn.reserve(r1 - r0);
    for (u32 rd = r0; rd < r1; ++rd)
        if ((u64)l <= off[rd + 1] - off[rd]) turn.push_back(Cursor{rd, 1, 0, 0, (int)l - 1, DS{0, 0, X.n}});
    while (!turn.empty()) {
        size_t kept = 0;
        for (size_t q = 0; q < turn.size(); ++q) {
            Cursor e = turn[q];
            if (!advance(X, seq + off[e.rd], (int)(off[e.rd + 1] - off[e.rd]), l, c, e, per[e.rd - r0])) continue;
            if (e.v.s != X.n) {
                const u64 p = e.u == 2 ? e.v.kr : e.v.k;
                prefetch_row(X, p);
                prefetch_row(X, p + e.v.s);
            }
            turn[kept++] = e;
        }
        turn.resize(kept);
    }
    for (auto &v : per) out.insert(out.end(), v.begin(), v.end());
}

// Algorithm 2, BatchLocate: all rows of the batch advance one level at a time
void batch_locate(const Index &X, const std::vector<u64> &rows, u32 *pos) {
    struct W { u64 k; u64 idx; u32 steps; };
    std::vector<W> E(rows.size()), E2;
    for (size_t q = 0; q < rows.size(); ++q) E[q] = W{rows[q], q, 0};
    while (!E.empty()) {
        E2.clear();
        for (const W &w : E) {
            if (w.k % X.r == 0) pos[w.idx] = (u32)(((u64)X.ssa[w.k / X.r] + w.steps) % X.n);
            else if (w.k == X.primary) pos[w.idx] = w.steps;   // S = 0
            else {
                const u64 nk = lf(X, w.k);
                prefetch_row(X, nk);
                E2.push_back(W{nk, w.idx, w.steps + 1});
            }
        }
        E.swap(E2);
    }
}

}  // namespace

extern "C" {

/* Index from the BWT (n bytes: 0 = $, 1..4 = A..T), the row of $ and the sampled suffix array
 * (ceil(n / r) u32 of S(x r)). */
void *cb_index_build(const u8 *bwt, u64 n, u64 primary, const u32 *ssa, u32 r, int threads) {
    Index *X = new Index;
    X->n = n;
    X->primary = primary;
    X->r = r;
    const u64 nb = n / 128 + 1;
    X->blk.assign(nb, Block{});
    std::vector<u64> cnt(nb * 4, 0);
    const int th = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for num_threads(th) schedule(static)
    for (u64 b = 0; b < nb; ++b) {
        Block &B = X->blk[b];
        for (u32 q = 0; q < 128; ++q) {
            const u64 x = b * 128 + q;
            if (x >= n) break;
            const u8 s = bwt[x];
            const u32 code = s == 0 ? 0u : (u32)(s - 1);
            B.w[q >> 5] |= (u64)code << (2 * (q & 31));
            if (s) ++cnt[b * 4 + code];
        }
    }
    u64 run[4] = {0, 0, 0, 0};
    for (u64 b = 0; b < nb; ++b)
        for (u32 a = 0; a < 4; ++a) {
            X->blk[b].cnt[a] = run[a];
            run[a] += cnt[b * 4 + a];
        }
    X->C[0] = 1;
    for (u32 a = 1; a < 4; ++a) X->C[a] = X->C[a - 1] + run[a - 1];
    X->ssa.assign(ssa, ssa + (n + r - 1) / r);
    // ds-intervals of all 10-mers: 10 BackwardExt steps from (0, 0, n), last base first
    const u64 nk = 1ULL << (2 * KTAB);
    X->kmer.assign(nk * 3, 0);
#pragma omp parallel for num_threads(th) schedule(static)
    for (u64 w = 0; w < nk; ++w) {
        DS v{0, 0, n};
        for (int t = (int)KTAB - 1; t >= 0 && v.s; --t) v = backward_ext(*X, v, (u32)(w >> (2 * t)) & 3u);
        X->kmer[3 * w] = v.k;
        X->kmer[3 * w + 1] = v.kr;
        X->kmer[3 * w + 2] = v.s;
    }
    return X;
}

void cb_index_free(void *x) { delete (Index *)x; }

struct CbResult {
    std::vector<Rec> smem;
    std::vector<u32> hits;
};

/* SMEMs (Algorithm 3, batches of `batch` reads per queue) and their hits (BatchLocate per batch)
 * for reads with codes 0..3 (4 = N); SMEMs with s > max_occ get no hits.  Returns a handle. */
void *cb_seed(void *x, const u8 *seq, const u64 *off, u32 nr, u32 l, u32 c, u32 max_occ, u32 batch, int threads) {
    const Index &X = *(Index *)x;
    if (batch == 0) batch = 4096;
    const u32 nbt = (nr + batch - 1) / batch;
    std::vector<std::vector<Rec>> recs(nbt);
    std::vector<std::vector<u32>> hits(nbt);
#pragma omp parallel for num_threads(threads > 0 ? threads : omp_get_max_threads()) schedule(dynamic, 1)
    for (u32 b = 0; b < nbt; ++b) {
        const u32 r0 = b * batch, r1 = std::min(nr, r0 + batch);
        batch_find_smem(X, seq, off, r0, r1, l, c, recs[b]);
        std::vector<u64> rows;
        for (const Rec &m : recs[b])
            if (m.s <= max_occ)
                for (u64 t = 0; t < m.s; ++t) rows.push_back(m.k + t);
        hits[b].resize(rows.size());
        batch_locate(X, rows, hits[b].data());
    }
    CbResult *R = new CbResult;
    for (u32 b = 0; b < nbt; ++b) {
        R->smem.insert(R->smem.end(), recs[b].begin(), recs[b].end());
        R->hits.insert(R->hits.end(), hits[b].begin(), hits[b].end());
    }
    return R;
}
u64 cb_result_nsmem(void *r) { return ((CbResult *)r)->smem.size(); }
u64 cb_result_nhits(void *r) { return ((CbResult *)r)->hits.size(); }
/* records as 6 u64 each (read, qbeg, qend, k, kr, s), then the hits */
void cb_result_get(void *r, u64 *smem, u32 *hits) {
    const CbResult &R = *(CbResult *)r;
    for (size_t q = 0; q < R.smem.size(); ++q) {
        const Rec &m = R.smem[q];
        u64 *o = smem + 6 * q;
        o[0] = m.read; o[1] = m.qbeg; o[2] = m.qend; o[3] = m.k; o[4] = m.kr; o[5] = m.s;
    }
    if (!R.hits.empty()) memcpy(hits, R.hits.data(), R.hits.size() * 4);
}
void cb_result_free(void *r) { delete (CbResult *)r; }

}  // extern "C"
