// Mate-rescue prefilter of Section 2.7 (mb_rescue_prefilter): for a read P and a reference window
// R, M_t = #{(i, j) : P[i, i+q) = R[j, j+q), j - i = t}, and the result is max_t M_t.
//
// One warp per (read, window) pair, bit-parallel along each diagonal.  The warp writes, for each
// base a, the bit masks P_a (bit i = [P[i] = a]) and R_a (bit j = [R[j] = a], behind a zero pad so
// that negative diagonals read zeros) into its slice of shared memory, by ballots.  Lane l takes
// the diagonals t = t0 + l, t0 + l + 32, ...; on diagonal t the word D_k = OR_a P_a[k] & (R_a
// shifted by t) has bit i set where P[i] = R[i+t] (an N is in no mask, so it matches nothing), a
// q-mer match at i is a run of q set bits starting at i (q - 1 shifted ANDs, the next word
// carried in), and M_t is the popcount of those run starts.  64 positions of a diagonal cost
// about 30 integer operations instead of 64 code compares.
#include <algorithm>
#include <vector>
#include "common.cuh"

namespace {

// 64 bits of the padded mask m starting at bit b
__device__ __forceinline__ u64 bits_at(const u64 *__restrict__ m, u32 b) {
    const u32 w = b >> 6, s = b & 63;
    const u64 lo = m[w];
    return s ? (lo >> s) | (m[w + 1] << (64 - s)) : lo;
}

// Words per base of a pair's masks: P (np words), R (pad np + nr + np + 1 words).
__host__ __device__ __forceinline__ u32 words_p(u32 m) { return (m + 63) / 64; }
__host__ __device__ __forceinline__ u32 words_r(u32 m, u32 w) { return 2 * words_p(m) + (w + 63) / 64 + 1; }

// masks of x (len bases) at bit offset `shift` of 4 arrays of `stride` words (already zero)
__device__ __forceinline__ void build_masks(const u8 *__restrict__ x, u32 len, u64 *__restrict__ M, u32 stride,
                                            u32 shift, u32 lane) {
    u32 *M32 = reinterpret_cast<u32 *>(M);
    for (u32 c = 0; c * 32 < len; ++c) {
        const u32 i = c * 32 + lane;
        const u32 b = i < len ? x[i] : 4u;
#pragma unroll
        for (u32 a = 0; a < 4; ++a) {
            const u32 bal = __ballot_sync(0xffffffffu, b == a);
            if (lane == a) M32[2 * stride * a + (shift >> 5) + c] = bal;   // shift is a multiple of 64
        }
    }
}

__global__ void k_qmer_diag_max(const u8 *__restrict__ reads, const u64 *__restrict__ roff,
                                const u8 *__restrict__ wins, const u64 *__restrict__ woff, u32 npairs, u32 q,
                                u32 slice_words, u32 *__restrict__ best) {
    extern __shared__ u64 sm[];
    const u32 lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    u64 *S = sm + (size_t)wib * slice_words;
    const u32 nw = (gridDim.x * blockDim.x) >> 5;
    for (u32 p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npairs; p += nw) {
        const u64 r0 = roff[p], w0 = woff[p];
        const u32 m = (u32)(roff[p + 1] - r0), w = (u32)(woff[p + 1] - w0);
        const u32 np = words_p(m), sr = words_r(m, w);
        u64 *Pm = S, *Rm = S + 4 * np;
        for (u32 k = lane; k < 4 * (np + sr); k += 32) S[k] = 0;
        __syncwarp();
        build_masks(reads + r0, m, Pm, np, 0, lane);
        build_masks(wins + w0, w, Rm, sr, 64 * np, lane);
        __syncwarp();
        const int mp = m >= q ? (int)(m - q + 1) : 0, wr = w >= q ? (int)(w - q + 1) : 0;
        u32 top = 0;
        if (mp > 0 && wr > 0) {
            for (int t = -(mp - 1) + (int)lane; t <= wr - 1; t += 32) {
                const u32 base = (u32)((int)(64 * np) + t);   // bit of R_a for j = t (>= 1)
                auto diag = [&](u32 k) -> u64 {
                    u64 d = 0;
#pragma unroll
                    for (u32 a = 0; a < 4; ++a) d |= Pm[a * np + k] & bits_at(Rm + a * sr, base + 64 * k);
                    return d;
                };
                u32 cnt = 0;
                u64 dn = diag(0);
                for (u32 k = 0; k < np; ++k) {
                    const u64 d = dn;
                    dn = k + 1 < np ? diag(k + 1) : 0;
                    u64 run = d;
                    for (u32 s = 1; s < q; ++s) run &= (d >> s) | (dn << (64 - s));
                    cnt += __popcll(run);
                }
                top = max(top, cnt);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
        if (lane == 0) best[p] = top;
        __syncwarp();   // the masks are rewritten for the next pair
    }
}

}  // namespace

extern "C" int mb_rescue_prefilter(const uint8_t *reads, const uint64_t *read_off, const uint8_t *wins,
                                   const uint64_t *win_off, uint32_t n_pairs, uint32_t q, void *stream,
                                   uint32_t *best) {
    if (!read_off || !win_off || !best || (n_pairs && (!reads || !wins))) {
        mb_set_error("mb_rescue_prefilter: null argument");
        return MB_ERR_ARG;
    }
    if (q == 0) q = 7;
    if (q > 15) {
        mb_set_error("mb_rescue_prefilter: q = %u, at most 15", q);
        return MB_ERR_ARG;
    }
    if (n_pairs == 0) return MB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the longest read and window size the shared-memory slices
    std::vector<u64> ro(n_pairs + 1), wo(n_pairs + 1);
    MB_CK(cudaMemcpyAsync(ro.data(), read_off, ro.size() * 8, cudaMemcpyDefault, st));
    MB_CK(cudaMemcpyAsync(wo.data(), win_off, wo.size() * 8, cudaMemcpyDefault, st));
    MB_CK(cudaStreamSynchronize(st));
    u64 mmax = 0, wmax = 0;
    for (u32 p = 0; p < n_pairs; ++p) {
        if (ro[p + 1] < ro[p] || wo[p + 1] < wo[p]) {
            mb_set_error("mb_rescue_prefilter: offsets decrease at pair %u", p);
            return MB_ERR_ARG;
        }
        mmax = std::max(mmax, ro[p + 1] - ro[p]);
        wmax = std::max(wmax, wo[p + 1] - wo[p]);
    }
    // mask words per warp: 4 bases x (P words + padded R words) of the longest read and window
    const u64 np = (mmax + 63) / 64, nr = (wmax + 63) / 64;
    const u64 slice = 4 * (np + 2 * np + nr + 1);
    const size_t per_warp = (size_t)slice * 8;
    int dev = 0, smem_max = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_warp > (size_t)smem_max) {
        mb_set_error("mb_rescue_prefilter: a read of %llu and a window of %llu bases need %zu bytes of "
                     "shared memory, more than %d",
                     (unsigned long long)mmax, (unsigned long long)wmax, per_warp, smem_max);
        return MB_ERR_ARG;
    }
    int warps = (int)std::min<size_t>(8, (size_t)smem_max / per_warp);
    const size_t smem = per_warp * warps;
    if (smem > 48 * 1024)
        MB_CK(cudaFuncSetAttribute(k_qmer_diag_max, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qmer_diag_max, warps * 32, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const u64 blocks = std::min<u64>((u64)sms * per_sm, ((u64)n_pairs + warps - 1) / warps);

    DevBuf br, bw, bro, bwo, bb;
    const void *dr, *dw, *dro, *dwo;
    MB_TRY(mb_stage_in(reads, ro[n_pairs], st, br, &dr));
    MB_TRY(mb_stage_in(wins, wo[n_pairs], st, bw, &dw));
    MB_TRY(mb_stage_in(read_off, ro.size() * 8, st, bro, &dro));
    MB_TRY(mb_stage_in(win_off, wo.size() * 8, st, bwo, &dwo));
    u32 *db = best;
    const bool bdev = mb_is_device_ptr(best);
    if (!bdev) {
        MB_TRY(bb.alloc((size_t)n_pairs * 4, st));
        db = bb.as<u32>();
    }
    KTimer kt("rescue", st);
    kt.start();
    k_qmer_diag_max<<<(unsigned)blocks, warps * 32, smem, st>>>((const u8 *)dr, (const u64 *)dro, (const u8 *)dw,
                                                                (const u64 *)dwo, n_pairs, q, (u32)slice, db);
    MB_KCHECK();
    kt.stop();
    if (!bdev) MB_CK(cudaMemcpyAsync(best, db, (size_t)n_pairs * 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    return MB_OK;
}
