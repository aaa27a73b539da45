// Mate-rescue prefilter of Section 2.6 (mb_rescue_prefilter): for a read P and a reference window
// R, M_t = #{(i, j) : P[i, i+q) = R[j, j+q), j - i = t}, and the result is max_t M_t.
//
// One warp per (read, window) pair.  The warp writes the q-mer codes of P and R into its slice of
// shared memory (a q-mer holding an N gets a code no other q-mer has), then each lane takes every
// 32nd diagonal t and counts the equal codes along it: lanes work on neighbouring diagonals, so
// at each step they read one code of P (a broadcast) and 32 consecutive codes of R (no bank
// conflict).  Integer compares only; no tensor-core form exists for diagonal counts.
#include <algorithm>
#include <vector>
#include "common.cuh"

namespace {

constexpr u32 BAD_P = 0xFFFFFFFFu, BAD_R = 0xFFFFFFFEu;   // q-mers with an N (q <= 15: codes < 2^30)

__device__ __forceinline__ void qmer_codes(const u8 *__restrict__ x, u32 len, u32 q, u32 bad, u32 *__restrict__ c,
                                           u32 lane) {
    const u32 nq = len >= q ? len - q + 1 : 0;
    for (u32 i = lane; i < nq; i += 32) {
        u32 v = 0, n = 0;
        for (u32 k = 0; k < q; ++k) {
            const u32 b = x[i + k];
            n |= b > 3 ? 1u : 0u;
            v = (v << 2) | (b & 3u);
        }
        c[i] = n ? bad : v;
    }
}

__global__ void k_qmer_diag_max(const u8 *__restrict__ reads, const u64 *__restrict__ roff,
                                const u8 *__restrict__ wins, const u64 *__restrict__ woff, u32 npairs, u32 q,
                                u32 cap_p, u32 cap_r, u32 *__restrict__ best) {
    extern __shared__ u32 sm[];
    const u32 lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    u32 *Pc = sm + (size_t)wib * (cap_p + cap_r), *Rc = Pc + cap_p;
    const u32 nw = (gridDim.x * blockDim.x) >> 5;
    for (u32 p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npairs; p += nw) {
        const u64 r0 = roff[p], w0 = woff[p];
        const u32 m = (u32)(roff[p + 1] - r0), w = (u32)(woff[p + 1] - w0);
        qmer_codes(reads + r0, m, q, BAD_P, Pc, lane);
        qmer_codes(wins + w0, w, q, BAD_R, Rc, lane);
        __syncwarp();
        const int mp = m >= q ? (int)(m - q + 1) : 0, wr = w >= q ? (int)(w - q + 1) : 0;
        u32 top = 0;
        if (mp > 0 && wr > 0) {
            // diagonal t = j - i runs from -(mp - 1) to wr - 1
            for (int t = -(mp - 1) + (int)lane; t <= wr - 1; t += 32) {
                const int i0 = t < 0 ? -t : 0, i1 = min(mp, wr - t);   // i in [i0, i1)
                u32 cnt = 0;
                for (int i = i0; i < i1; ++i) cnt += Pc[i] == Rc[i + t] ? 1u : 0u;
                top = max(top, cnt);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
        if (lane == 0) best[p] = top;
        __syncwarp();   // the codes are rewritten for the next pair
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
    const u32 cap_p = (u32)std::max<u64>(mmax, 1), cap_r = (u32)std::max<u64>(wmax, 1);
    const size_t per_warp = ((size_t)cap_p + cap_r) * 4;
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
                                                                (const u64 *)dwo, n_pairs, q, cap_p, cap_r, db);
    MB_KCHECK();
    kt.stop();
    if (!bdev) MB_CK(cudaMemcpyAsync(best, db, (size_t)n_pairs * 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));
    return MB_OK;
}
