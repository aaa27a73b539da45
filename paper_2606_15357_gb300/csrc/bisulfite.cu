// Section 2.9 on the GPU: the T-to-C split of bisulfite seed matches (mb_bs_split).
//
// A seed found on the 3-base index matches the converted read against the converted reference,
// so a read C over a reference T (read 1, C->T) or a read G over a reference A (read 2, G->A)
// matches there although the original bases differ.  Each kept hit of a seed is compared base by
// base with the original reference under it and cut at every such position; the pieces of at
// least min_len bases are the output.  Two passes over the hits (count, then write at the
// scanned offsets), one thread per hit.
#include "common.cuh"

namespace {

// the record owning hit h: the last record whose first hit is at or before h
__device__ __forceinline__ u64 record_of(const mb_smem *__restrict__ sm, u64 nsm, u64 h) {
    u64 a = 0, b = nsm;
    while (b - a > 1) {
        const u64 mid = (a + b) >> 1;
        if (__ldg(&sm[mid].hit_off) <= h) a = mid;
        else b = mid;
    }
    return a;
}

__device__ __forceinline__ u32 comp_code(u32 b) { return b < 4 ? 3u - b : 4u; }

// Calls emit(a, b) for every piece [a, b) (offsets in the seed) of hit h of record x at text
// position pos, in order.  M = |R|; the text is CT(R) GA(R) rc(GA(R)) rc(CT(R)) $.  A hit that
// does not lie inside one copy gives nothing.
template <class Emit>
__device__ __forceinline__ void pieces(const u8 *__restrict__ ref, u64 M, const u8 *__restrict__ seq,
                                       const u64 *__restrict__ off, const u8 *__restrict__ mate, const mb_smem &x,
                                       u64 pos, u32 min_len, Emit &emit) {
    const u32 L = x.qend - x.qbeg;
    const u64 g = pos / M, q = pos - g * M;
    if (L == 0 || g > 3 || (pos + L - 1) / M != g) return;
    const u32 mt = mate ? mate[x.read] : 0u;
    if (mt != 1 && mt != 2) {                 // unconverted read: no cut
        if (L >= min_len) emit(0u, L);
        return;
    }
    const u32 cut_read = mt == 1 ? 1u : 2u;   // read C (read 1) or read G (read 2)
    const u32 cut_ref = mt == 1 ? 3u : 0u;    // over reference T or A
    const u8 *__restrict__ P = seq + off[x.read] + x.qbeg;
    u32 start = 0;
    for (u32 t = 0; t < L; ++t) {
        if (P[t] != cut_read) continue;
        const u32 r = g < 2 ? (u32)ref[q + t] : comp_code(ref[M - 1 - (q + t)]);
        if (r != cut_ref) continue;
        if (t - start >= min_len) emit(start, t);
        start = t + 1;
    }
    if (L - start >= min_len) emit(start, L);
}

struct CountEmit {
    u64 n = 0;
    __device__ __forceinline__ void operator()(u32, u32) { ++n; }
};

struct WriteEmit {
    mb_piece *out;
    u64 at, cap, hit;
    u32 read, qbeg, pos;
    __device__ __forceinline__ void operator()(u32 a, u32 b) {
        if (at < cap) out[at] = mb_piece{hit, read, qbeg + a, qbeg + b, pos + a};
        ++at;
    }
};

__global__ void k_split_count(const mb_smem *__restrict__ sm, u64 nsm, const u32 *__restrict__ hits,
                              const u8 *__restrict__ keep, u64 nh, const u8 *__restrict__ ref, u64 M,
                              const u8 *__restrict__ seq, const u64 *__restrict__ off, const u8 *__restrict__ mate,
                              u32 min_len, u64 *__restrict__ cnt) {
    for (u64 h = blockIdx.x * (u64)blockDim.x + threadIdx.x; h < nh; h += (u64)gridDim.x * blockDim.x) {
        CountEmit e;
        if (!keep || keep[h]) {
            const mb_smem x = sm[record_of(sm, nsm, h)];
            pieces(ref, M, seq, off, mate, x, hits[h], min_len, e);
        }
        cnt[h] = e.n;
    }
}

__global__ void k_split_write(const mb_smem *__restrict__ sm, u64 nsm, const u32 *__restrict__ hits,
                              const u8 *__restrict__ keep, u64 nh, const u8 *__restrict__ ref, u64 M,
                              const u8 *__restrict__ seq, const u64 *__restrict__ off, const u8 *__restrict__ mate,
                              u32 min_len, const u64 *__restrict__ at, mb_piece *__restrict__ out, u64 cap) {
    for (u64 h = blockIdx.x * (u64)blockDim.x + threadIdx.x; h < nh; h += (u64)gridDim.x * blockDim.x) {
        if (keep && !keep[h]) continue;
        const mb_smem x = sm[record_of(sm, nsm, h)];
        WriteEmit e{out, at[h], cap, h, x.read, x.qbeg, hits[h]};
        pieces(ref, M, seq, off, mate, x, hits[h], min_len, e);
    }
}

}  // namespace

extern "C" int mb_bs_split(const mb_index *idx, const uint8_t *ref, const uint8_t *seq, const uint64_t *off,
                           uint32_t n_reads, const uint8_t *mate, const mb_smem *smem, uint64_t n_smem,
                           const uint32_t *hits, const uint8_t *keep, uint64_t n_hits, const mb_opts *opts,
                           void *stream, mb_piece *out, uint64_t cap, uint64_t *n_out) {
    if (!idx || !n_out || (n_hits && (!ref || !seq || !off || !smem || !hits || !n_smem))) {
        mb_set_error("mb_bs_split: null argument");
        return MB_ERR_ARG;
    }
    *n_out = 0;
    if (!(mb_index_flags(idx) & MB_BS3)) {
        mb_set_error("mb_bs_split: the index is not a bisulfite (MB_BS3) index");
        return MB_ERR_ARG;
    }
    if (n_hits == 0) return MB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    u64 n = 0, prim = 0, r3 = 0;
    MB_TRY(mb_index_info(idx, &n, &prim, &r3));
    const u64 M = r3 / 2;   // the index holds CT(R) GA(R): |R3| = 2 |R|
    const u32 min_len = opts && opts->min_len ? opts->min_len : 19;

    u64 o_last = 0;
    MB_CK(cudaMemcpyAsync(&o_last, off + n_reads, 8, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    DevBuf bref, bseq, boff, bmate, bsm, bhits, bkeep, bcnt, btmp, bout;
    const void *dref, *dseq, *doff, *dmate = nullptr, *dsm, *dhits, *dkeep = nullptr;
    MB_TRY(mb_stage_in(ref, M, st, bref, &dref));
    MB_TRY(mb_stage_in(seq, o_last, st, bseq, &dseq));
    MB_TRY(mb_stage_in(off, ((size_t)n_reads + 1) * 8, st, boff, &doff));
    if (mate) MB_TRY(mb_stage_in(mate, n_reads, st, bmate, &dmate));
    MB_TRY(mb_stage_in(smem, n_smem * sizeof(mb_smem), st, bsm, &dsm));
    MB_TRY(mb_stage_in(hits, n_hits * 4, st, bhits, &dhits));
    if (keep) MB_TRY(mb_stage_in(keep, n_hits, st, bkeep, &dkeep));
    MB_TRY(bcnt.alloc(n_hits * 8 + 64, st));
    u64 *cnt = bcnt.as<u64>(), *dtotal = cnt + n_hits;
    const unsigned G = grid_for(n_hits, 256);
    k_split_count<<<G, 256, 0, st>>>((const mb_smem *)dsm, n_smem, (const u32 *)dhits, (const u8 *)dkeep, n_hits,
                                     (const u8 *)dref, M, (const u8 *)dseq, (const u64 *)doff, (const u8 *)dmate,
                                     min_len, cnt);
    MB_KCHECK();
    MB_TRY(btmp.alloc(scan_tmp_bytes(n_hits), st));
    MB_TRY(scan_exclusive_u64(cnt, cnt, n_hits, dtotal, btmp.p, st));
    u64 total = 0;
    MB_CK(cudaMemcpyAsync(&total, dtotal, 8, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    *n_out = total;
    if (total > cap) return MB_ERR_CAPACITY;
    if (total == 0) return MB_OK;
    if (!out) return MB_ERR_ARG;
    mb_piece *dout = out;
    const bool odev = mb_is_device_ptr(out);
    if (!odev) {
        MB_TRY(bout.alloc(total * sizeof(mb_piece), st));
        dout = bout.as<mb_piece>();
    }
    k_split_write<<<G, 256, 0, st>>>((const mb_smem *)dsm, n_smem, (const u32 *)dhits, (const u8 *)dkeep, n_hits,
                                     (const u8 *)dref, M, (const u8 *)dseq, (const u64 *)doff, (const u8 *)dmate,
                                     min_len, cnt, dout, total);
    MB_KCHECK();
    if (!odev) MB_CK(cudaMemcpyAsync(out, dout, total * sizeof(mb_piece), cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    return MB_OK;
}
