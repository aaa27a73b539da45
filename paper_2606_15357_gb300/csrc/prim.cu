// Device primitives used by the index builder and the seeding pipeline: prefix scans and a
// stable LSD radix sort of (u64 key, u32 value) pairs.
#include "common.cuh"

namespace {

constexpr int SCAN_T = 256;      // threads per scan block
constexpr int SCAN_I = 16;       // items per thread
constexpr size_t SCAN_TILE = (size_t)SCAN_T * SCAN_I;

struct OpSum {
    template <class T> __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
    template <class T> static __device__ __forceinline__ T id() { return T(0); }
};
struct OpMax {
    template <class T> __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
    template <class T> static __device__ __forceinline__ T id() { return T(0); }
};

template <class T, class Op>
__device__ __forceinline__ T warp_incl(T v, Op op) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v = op(v, o);
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix and the total.
template <class T, class Op>
__device__ __forceinline__ T block_excl(T v, T &total, Op op) {
    __shared__ T ws[SCAN_T / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = warp_incl(v, op);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_T / 32 ? ws[lane] : Op::template id<T>();
        T wi = warp_incl(w, op);
        if (lane < SCAN_T / 32) ws[lane] = wi;   // inclusive over warps
    }
    __syncthreads();
    T warp_pre = warp == 0 ? Op::template id<T>() : ws[warp - 1];
    total = ws[SCAN_T / 32 - 1];
    T ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = Op::template id<T>();
    __syncthreads();
    return op(warp_pre, ex);
}

template <class T, class Op>
__global__ void k_scan_reduce(const T *__restrict__ in, size_t n, T *__restrict__ part, Op op) {
    size_t base = blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_I;
    T acc = Op::template id<T>();
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i)
        if (base + i < n) acc = op(acc, in[base + i]);
    T tot;
    block_excl(acc, tot, op);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Scans one tile; carry = scanned partial of this tile (exclusive), or identity for one tile.
template <class T, class Op, bool INCL>
__global__ void k_scan_apply(const T *in, T *out, size_t n, const T *__restrict__ carry, T *total, Op op) {
    size_t base = blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_I;
    T v[SCAN_I];
    T acc = Op::template id<T>();
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        v[i] = base + i < n ? in[base + i] : Op::template id<T>();
        acc = op(acc, v[i]);
    }
    T tot;
    T pre = block_excl(acc, tot, op);
    T c = carry ? carry[blockIdx.x] : Op::template id<T>();
    pre = op(c, pre);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        T nx = op(pre, v[i]);
        if (base + i < n) out[base + i] = INCL ? nx : pre;
        pre = nx;
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = op(c, tot);
}

size_t level_blocks(size_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

template <class T, class Op, bool INCL>
int scan_impl(const T *in, T *out, size_t n, void *tmp, cudaStream_t st, Op op) {
    if (n == 0) return MB_OK;
    size_t nb = level_blocks(n);
    if (nb == 1) {
        k_scan_apply<T, Op, INCL><<<1, SCAN_T, 0, st>>>(in, out, n, nullptr, nullptr, op);
        MB_KCHECK();
        return MB_OK;
    }
    T *part = (T *)tmp;
    void *rest = (void *)((char *)tmp + ((nb * sizeof(u64) + 255) & ~(size_t)255));
    k_scan_reduce<T, Op><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, part, op);
    MB_KCHECK();
    // exclusive scan of the tile sums gives each tile's carry
    MB_TRY((scan_impl<T, Op, false>(part, part, nb, rest, st, op)));
    k_scan_apply<T, Op, INCL><<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, part, nullptr, op);
    MB_KCHECK();
    return MB_OK;
}

template <class T>
__global__ void k_copy_one(const T *src, T *dst) { *dst = *src; }
template <class T>
__global__ void k_add_one(const T *src, T *dst) { *dst += *src; }

// exclusive sum; total = last input + last output (the last input is saved first so that the
// scan may run in place)
template <class T>
int scan_excl_total(const T *in, T *out, size_t n, T *total, void *tmp, cudaStream_t st) {
    if (n == 0) {
        if (total) MB_CK(cudaMemsetAsync(total, 0, sizeof(T), st));
        return MB_OK;
    }
    if (total) {
        k_copy_one<T><<<1, 1, 0, st>>>(in + n - 1, total);
        MB_KCHECK();
    }
    MB_TRY((scan_impl<T, OpSum, false>(in, out, n, tmp, st, OpSum())));
    if (total) {
        k_add_one<T><<<1, 1, 0, st>>>(out + n - 1, total);
        MB_KCHECK();
    }
    return MB_OK;
}

}  // namespace

size_t scan_tmp_bytes(size_t n) {
    size_t b = 0;
    size_t nb = level_blocks(n);
    while (nb > 1) {
        b += ((nb * sizeof(u64) + 255) & ~(size_t)255);
        nb = level_blocks(nb);
    }
    return b + 256;
}

int scan_exclusive_u64(const u64 *in, u64 *out, size_t n, u64 *total, void *tmp, cudaStream_t st) {
    return scan_excl_total<u64>(in, out, n, total, tmp, st);
}

int scan_exclusive_u32(const u32 *in, u32 *out, size_t n, u32 *total, void *tmp, cudaStream_t st) {
    return scan_excl_total<u32>(in, out, n, total, tmp, st);
}

int scan_inclusive_max_u32(const u32 *in, u32 *out, size_t n, void *tmp, cudaStream_t st) {
    return scan_impl<u32, OpMax, true>(in, out, n, tmp, st, OpMax());
}

// ============================================================================ radix sort
namespace {
constexpr int RS_T = 256;        // threads (8 warps)
constexpr int RS_I = 32;         // iterations of 32 items per warp
constexpr size_t RS_TILE = (size_t)RS_T * RS_I;

// n_dev (device, may be null): the number of items to sort when it is below n (the tiles past it
// count nothing and move nothing).
__device__ __forceinline__ size_t items(size_t n, const u64 *n_dev) { return n_dev && *n_dev < n ? (size_t)*n_dev : n; }

__global__ void __launch_bounds__(RS_T) k_radix_up(const u64 *__restrict__ keys, size_t n, const u64 *n_dev, int shift,
                                                   u32 mask, u32 *__restrict__ hist, size_t tiles) {
    __shared__ u32 h[256];
    n = items(n, n_dev);
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int it = 0; it < RS_I; ++it) {
        size_t idx = base + (size_t)it * RS_T + threadIdx.x;
        if (idx < n) atomicAdd(&h[(u32)(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Each warp owns a contiguous run of 32*RS_I items of the tile; items keep their order inside
// a warp (iteration-major, lane-minor), warps keep theirs inside the tile, tiles theirs inside
// a digit: the scatter is stable.
__global__ void __launch_bounds__(RS_T) k_radix_down(const u64 *__restrict__ keys, const u32 *__restrict__ vals,
                                                     u64 *__restrict__ okeys, u32 *__restrict__ ovals, size_t n,
                                                     const u64 *n_dev, int shift, u32 mask,
                                                     const u32 *__restrict__ offs, size_t tiles) {
    __shared__ u32 wh[RS_T / 32][256];
    n = items(n, n_dev);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (RS_T / 32) * 256; i += RS_T) (&wh[0][0])[i] = 0;
    __syncthreads();
    const size_t base = blockIdx.x * RS_TILE + (size_t)warp * 32 * RS_I;
    for (int it = 0; it < RS_I; ++it) {
        size_t idx = base + (size_t)it * 32 + lane;
        bool ok = idx < n;
        u32 d = ok ? ((u32)(keys[idx] >> shift) & mask) : 0xFFFFFFFFu;
        u32 peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) wh[warp][d] += __popc(peers);
    }
    __syncthreads();
    {
        u32 d = threadIdx.x;
        u32 run = offs[(size_t)d * tiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) {
            u32 t = wh[w][d];
            wh[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    const u32 lt = (1u << lane) - 1u;
    for (int it = 0; it < RS_I; ++it) {
        size_t idx = base + (size_t)it * 32 + lane;
        bool ok = idx < n;
        u64 k = ok ? keys[idx] : 0;
        u32 v = ok ? vals[idx] : 0;
        u32 d = ok ? ((u32)(k >> shift) & mask) : 0xFFFFFFFFu;
        u32 peers = __match_any_sync(0xffffffffu, d);
        u32 rank = __popc(peers & lt);
        u32 b = ok ? wh[warp][d] : 0;
        if (ok) {
            okeys[b + rank] = k;
            ovals[b + rank] = v;
        }
        __syncwarp();
        if (ok && rank == 0) wh[warp][d] = b + __popc(peers);
        __syncwarp();
    }
}
}  // namespace

size_t radix_tmp_bytes(size_t n) {
    size_t tiles = (n + RS_TILE - 1) / RS_TILE;
    size_t h = ((256 * tiles * sizeof(u32)) + 255) & ~(size_t)255;
    return h + scan_tmp_bytes(256 * tiles);
}

int radix_sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, size_t n, const BitRange *ranges,
                     int nranges, void *tmp, cudaStream_t st, const u64 *n_dev) {
    if (n <= 1) return MB_OK;
    if (n >= (1ULL << 32)) {
        mb_set_error("radix_sort_pairs: %zu items exceed 2^32-1", n);
        return MB_ERR_ARG;
    }
    size_t tiles = (n + RS_TILE - 1) / RS_TILE;
    u32 *hist = (u32 *)tmp;
    void *stmp = (char *)tmp + (((256 * tiles * sizeof(u32)) + 255) & ~(size_t)255);
    u64 *ka = keys, *kb = keys_alt;
    u32 *va = vals, *vb = vals_alt;
    int passes = 0;
    for (int r = 0; r < nranges; ++r) {
        for (int sh = ranges[r].lo; sh < ranges[r].hi; sh += 8) {
            int w = ranges[r].hi - sh < 8 ? ranges[r].hi - sh : 8;
            u32 mask = (1u << w) - 1u;
            k_radix_up<<<(unsigned)tiles, RS_T, 0, st>>>(ka, n, n_dev, sh, mask, hist, tiles);
            MB_KCHECK();
            MB_TRY(scan_exclusive_u32(hist, hist, 256 * tiles, nullptr, stmp, st));
            k_radix_down<<<(unsigned)tiles, RS_T, 0, st>>>(ka, va, kb, vb, n, n_dev, sh, mask, hist, tiles);
            MB_KCHECK();
            u64 *tk = ka; ka = kb; kb = tk;
            u32 *tv = va; va = vb; vb = tv;
            ++passes;
        }
    }
    if (passes & 1) {
        MB_CK(cudaMemcpyAsync(keys, ka, n * sizeof(u64), cudaMemcpyDeviceToDevice, st));
        MB_CK(cudaMemcpyAsync(vals, va, n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
    }
    return MB_OK;
}
