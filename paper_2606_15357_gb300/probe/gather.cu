// Random-gather ceiling of this GPU's memory system, for the roofline of the seeding kernels.
// Measurement utility only (no counterpart in the paper); used by bench.py.
//
//   mode 0: independent random block reads, 8 in flight per thread (bandwidth ceiling)
//   mode 1: dependent chains: each read's address comes from the data just read, the access
//           pattern of an LF-walk (latency-bound ceiling at full occupancy)
//   mode 2: as mode 1 with loads cached in L2 only (ld.global.cg)
// Blocks are 64 bytes (two 256-bit loads) or 32 bytes (one), at random block-aligned places of
// a buffer of `bytes` bytes (fewer than 2^32 blocks).
#include <cuda_runtime.h>
#include <stdint.h>

typedef uint64_t u64;

namespace {

__device__ __forceinline__ u64 mix(u64 z) {   // 64-bit hash: only used to fill the buffer
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// 32-bit hash (a few integer ops) and block index = high half of hash * number of blocks, so the
// probe's own arithmetic stays far below its memory traffic
__device__ __forceinline__ uint32_t h32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    return x ^ (x >> 16);
}

// CG = false: non-coherent path, cached in L1; CG = true: cached in L2 only
template <int BYTES, bool CG = false>
__device__ __forceinline__ u64 ld_block(const u64 *p) {
    u64 a, b, c, d;
    if (CG) asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
    else asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
    u64 r = a ^ b ^ c ^ d;
    if (BYTES == 64) {
        if (CG) asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 4));
        else asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 4));
        r ^= a ^ b ^ c ^ d;
    }
    return r;
}

__global__ void k_fill(u64 *buf, u64 words) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < words; i += (u64)gridDim.x * blockDim.x)
        buf[i] = mix(i + 12345);
}

template <int BYTES>
__global__ void __launch_bounds__(256) k_indep(const u64 *buf, u64 nblocks, unsigned iters, u64 *sink) {
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    u64 acc = 0;
    for (unsigned it = 0; it < iters; it += 8) {
        u64 idx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) idx[u] = __umulhi(h32((uint32_t)tid * 0x9E3779B9u + it * 8 + u), (uint32_t)nblocks);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= ld_block<BYTES>(buf + idx[u] * (BYTES / 8));
    }
    if (acc == 0x1234567) sink[tid & 1023] = acc;
}

template <int BYTES, bool CG = false>
__global__ void __launch_bounds__(256) k_chain(const u64 *buf, u64 nblocks, unsigned iters, u64 *sink) {
    const u64 tid = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    u64 idx = __umulhi(h32((uint32_t)tid), (uint32_t)nblocks);
    for (unsigned it = 0; it < iters; ++it)
        idx = __umulhi(h32((uint32_t)ld_block<BYTES, CG>(buf + idx * (BYTES / 8)) ^ it), (uint32_t)nblocks);
    if (idx == 0x1234567) sink[tid & 1023] = idx;
}

}  // namespace

// Returns the achieved rate in GB/s (bytes actually requested: BYTES per read), or a negative
// value on a CUDA error.  `ms` receives the kernel time.
extern "C" double mb_probe_gather(uint64_t bytes, int mode, int block_bytes, unsigned iters, float *ms) {
    if (block_bytes != 32 && block_bytes != 64) return -3;
    if (bytes / block_bytes >= (1ull << 32)) return -3;
    u64 *buf = nullptr, *sink = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return -1;
    if (cudaMalloc(&sink, 1024 * 8) != cudaSuccess) { cudaFree(buf); return -1; }
    const u64 words = bytes / 8, nblocks = bytes / block_bytes;
    k_fill<<<2048, 256>>>(buf, words);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *k = mode == 0 ? (block_bytes == 64 ? (const void *)k_indep<64> : (const void *)k_indep<32>)
                              : (block_bytes == 64 ? (const void *)k_chain<64> : (const void *)k_chain<32>);
    if (mode == 2) k = block_bytes == 64 ? (const void *)k_chain<64, true> : (const void *)k_chain<32, true>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 256, 0);
    const unsigned grid = (unsigned)(sms * (per > 0 ? per : 1));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float t = 0;
    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
        cudaEventRecord(a);
        if (mode == 0 && block_bytes == 64) k_indep<64><<<grid, 256>>>(buf, nblocks, iters, sink);
        else if (mode == 0) k_indep<32><<<grid, 256>>>(buf, nblocks, iters, sink);
        else if (mode == 2 && block_bytes == 64) k_chain<64, true><<<grid, 256>>>(buf, nblocks, iters, sink);
        else if (mode == 2) k_chain<32, true><<<grid, 256>>>(buf, nblocks, iters, sink);
        else if (block_bytes == 64) k_chain<64><<<grid, 256>>>(buf, nblocks, iters, sink);
        else k_chain<32><<<grid, 256>>>(buf, nblocks, iters, sink);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&t, a, b);
    }
    const bool ok = cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(sink);
    if (!ok) return -2;
    if (ms) *ms = t;
    const double reads = (double)grid * 256.0 * (double)iters;
    return reads * block_bytes / (t * 1e-3) / 1e9;
}
