// Internal definitions shared by the CUDA translation units of libminibwa_gpu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include "minibwa_gpu.h"

typedef uint64_t u64;
typedef uint32_t u32;
typedef uint8_t u8;

// ----------------------------------------------------------------------------- error plumbing
void mb_set_error(const char *fmt, ...);
#define MB_CK(call)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            mb_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));  \
            return e_ == cudaErrorMemoryAllocation ? MB_ERR_NOMEM : MB_ERR_CUDA;              \
        }                                                                                     \
    } while (0)
#define MB_TRY(expr)                 \
    do {                             \
        int r_ = (expr);             \
        if (r_ != MB_OK) return r_;  \
    } while (0)

// Stream-ordered device buffer owned by host code.  Freed on the stream it was made on.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t b, cudaStream_t s) {
        release();
        st = s;
        bytes = b;
        if (b == 0) return MB_OK;
        cudaError_t e = cudaMallocAsync(&p, b, s);
        if (e != cudaSuccess) {
            p = nullptr;
            mb_set_error("cudaMallocAsync(%zu): %s", b, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? MB_ERR_NOMEM : MB_ERR_CUDA;
        }
        return MB_OK;
    }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return (T *)p; }
};

bool mb_is_device_ptr(const void *p);

// launch bookkeeping: every kernel launch site calls MB_KCHECK() right after <<<...>>>
void mb_count_launch();
#define MB_KCHECK()                  \
    do {                             \
        MB_CK(cudaGetLastError());   \
        mb_count_launch();           \
    } while (0)

// CUDA-event timing of one kernel launch when profiling is on (see mb_profile_enable)
struct KTimer {
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(const char *n, cudaStream_t s);
    void start();
    void stop();
    ~KTimer();   // after the stream was synchronized: accumulates the elapsed time
};

// device-side work counters (index into the array handed to kernels in counting mode)
enum { WC_EXT_STEPS = 0, WC_EXT_BLOCKS = 1, WC_KMER = 2, WC_LF_STEPS = 3, WC_SA_READS = 4, WC_N = 5 };
u64 *mb_work_counter_buf(cudaStream_t st);   // device array of WC_N u64 (zeroed on first use)

// Stage a host-or-device input on the device: returns a device pointer (the input itself when
// it already is one, else a copy in `buf`).
int mb_stage_in(const void *src, size_t bytes, cudaStream_t st, DevBuf &buf, const void **dev);

// ----------------------------------------------------------------------------- index layout
// One occurrence block per 128 BWT rows (Section 2.2): the counts of A, C, G, T in B[0, 128b)
// as four u64, then the 128 symbols of B[128b, 128b+128) as four u64 words of 2-bit codes,
// row q of the block in word q/32 at bits 2*(q%32).  The $ row (primary) is stored as A and
// excluded from the counts.
struct __align__(64) OccBlock {
    u64 cnt[4];
    u64 w[4];
};

// Index view passed to kernels by value.
struct DevIndex {
    const OccBlock *occ;
    const u32 *ssa;     // S(x*r)
    const u32 *kmer;    // (k, kr, s) of every k-mer, first symbol most significant
    u64 n;              // |T|
    u64 primary;        // row with S = 0
    u64 C[4];           // C[a] = #{i : B[i] < a}, a = A,C,G,T
    u64 nblocks;
    u32 r;              // SA sample rate
    u32 kmer_k;
};

struct mb_index_impl;

// ----------------------------------------------------------------------------- device helpers
// Counts of A,C,G,T and of $ in B[0, x), from the block of row x.
struct Occ4 {
    u64 c[4];
    u32 dollar;
};

struct BlockVals {
    ulonglong2 c01, c23, w01, w23;
};
__device__ __forceinline__ BlockVals load_block(const OccBlock *__restrict__ blk) {
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(blk);
    BlockVals v;
    v.c01 = __ldg(p + 0);
    v.c23 = __ldg(p + 1);
    v.w01 = __ldg(p + 2);
    v.w23 = __ldg(p + 3);
    return v;
}

__device__ __forceinline__ void occ_from_vals(const BlockVals &v, u64 x, u64 primary, Occ4 &o) {
    u32 m = (u32)(x & 127);
    u64 w[4] = {v.w01.x, v.w01.y, v.w23.x, v.w23.y};
    u32 nl = 0, nh = 0, nt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int take = (int)m - 32 * q;
        take = take < 0 ? 0 : (take > 32 ? 32 : take);
        u64 mask = take == 32 ? ~0ULL : ((1ULL << (2 * take)) - 1);
        u64 y = w[q] & mask;
        u64 lo = y & 0x5555555555555555ULL, hi = (y >> 1) & 0x5555555555555555ULL;
        nl += __popcll(lo);
        nh += __popcll(hi);
        nt += __popcll(lo & hi);
    }
    // symbol codes: A=00 C=01 G=10 T=11 (low bit first)
    u32 cT = nt, cC = nl - nt, cG = nh - nt, cA = m - cC - cG - cT;
    u64 bstart = x & ~127ULL;
    u32 d = (primary >= bstart && primary < x) ? 1u : 0u;
    o.c[0] = v.c01.x + cA - d;
    o.c[1] = v.c01.y + cC;
    o.c[2] = v.c23.x + cG;
    o.c[3] = v.c23.y + cT;
    o.dollar = primary < x ? 1u : 0u;
}

// symbol (0..3) stored at row x of its block ($ reads as A)
__device__ __forceinline__ u32 sym_from_vals(const BlockVals &v, u64 x) {
    u32 q = (u32)(x & 127);
    u64 w = q < 64 ? ((q & 32) ? v.w01.y : v.w01.x) : ((q & 32) ? v.w23.y : v.w23.x);
    return (u32)(w >> (2 * (q & 31))) & 3u;
}

__device__ __forceinline__ void occ_from_block(const OccBlock *__restrict__ blk, u64 x, u64 primary, Occ4 &o) {
    occ_from_vals(load_block(blk), x, primary, o);
}

__device__ __forceinline__ void occ_at(const DevIndex &I, u64 x, Occ4 &o) {
    occ_from_block(I.occ + (x >> 7), x, I.primary, o);
}

// Algorithm 1 in one step.  Extends the interval (p, q, s) of P on the side of p by symbol a
// (0..3): p is lo of the strand being extended backwards, q is lo of the other strand.
//   s'  = #a in B[p, p+s)
//   p'  = C[a] + #a in B[0, p)
//   q'  = q + #{ $ or symbols > a } in B[p, p+s)
// BackwardExt((k,k',s), a) is (p,q) = (k,k'); ForwardExt((k,k',s), a) is (p,q) = (k',k) with
// the complement of a.
struct Ext {
    u64 p, q, s;
};
// x[a] for a in 0..3 without dynamic indexing (which would go through local memory)
__device__ __forceinline__ u64 sel4(u32 a, u64 x0, u64 x1, u64 x2, u64 x3) {
    return a < 2 ? (a == 0 ? x0 : x1) : (a == 2 ? x2 : x3);
}
__device__ __forceinline__ Ext extend_from(const DevIndex &I, const Occ4 &lo, const Occ4 &hi, u64 q,
                                           u32 a) {
    u64 d0 = hi.c[0] - lo.c[0], d1 = hi.c[1] - lo.c[1], d2 = hi.c[2] - lo.c[2], d3 = hi.c[3] - lo.c[3];
    u64 dd = hi.dollar - lo.dollar;
    u64 gt = dd + (a < 3 ? d3 : 0) + (a < 2 ? d2 : 0) + (a < 1 ? d1 : 0);
    Ext e;
    e.s = sel4(a, d0, d1, d2, d3);
    e.p = sel4(a, I.C[0] + lo.c[0], I.C[1] + lo.c[1], I.C[2] + lo.c[2], I.C[3] + lo.c[3]);
    e.q = q + gt;
    return e;
}

__device__ __forceinline__ Ext extend(const DevIndex &I, u64 p, u64 q, u64 s, u32 a) {
    Occ4 lo, hi;
    occ_at(I, p, lo);
    occ_at(I, p + s, hi);
    return extend_from(I, lo, hi, q, a);
}

// splitmix64 output function; bits 63..62 give the base replacing an ambiguous reference base.
__host__ __device__ __forceinline__ u64 mb_mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// ----------------------------------------------------------------------------- primitives
// Exclusive prefix sum of n values (in place allowed).  *total (device, may be null) receives
// the sum.  Uses `tmp` (device) of at least scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(size_t n);
int scan_exclusive_u64(const u64 *in, u64 *out, size_t n, u64 *total, void *tmp, cudaStream_t st);
int scan_exclusive_u32(const u32 *in, u32 *out, size_t n, u32 *total, void *tmp, cudaStream_t st);
// Inclusive prefix maximum of u32 values (in place allowed).
int scan_inclusive_max_u32(const u32 *in, u32 *out, size_t n, void *tmp, cudaStream_t st);

// Stable LSD radix sort of (key, val) pairs by the key bits in [lo_bit, hi_bit) of each digit
// range given.  Sorted output ends in (keys, vals); (keys_alt, vals_alt) are scratch of the
// same size.
struct BitRange {
    int lo, hi;
};
size_t radix_tmp_bytes(size_t n);
int radix_sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, size_t n, const BitRange *ranges,
                     int nranges, void *tmp, cudaStream_t st);

inline unsigned grid_for(size_t n, unsigned block, unsigned cap = 152u * 64u) {
    size_t g = (n + block - 1) / block;
    if (g > cap) g = cap;
    if (g == 0) g = 1;
    return (unsigned)g;
}
