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

// Keep freed stream-ordered memory in the device's pool between calls (the default threshold of 0
// returns it to the CUDA driver at every synchronization, so each call would map its scratch again).
void mb_keep_pool_memory();

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
        mb_keep_pool_memory();
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
// MB_ERR_ARG (with a message naming `what`) when device memory [p, p + bytes) passes the end of the
// device allocation holding p; MB_OK for host memory, null or empty spans.
int mb_check_span(const void *p, u64 bytes, const char *what);

// Device error word: set by kernels whose input fails a check (the access is skipped, never
// issued); the host returns MB_ERR_DEVICE_CHECK when it is not zero.
enum { DEVCHK_OFFSETS = 1u, DEVCHK_RECORD = 2u, DEVCHK_BOUNDS = 4u };

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
enum {
    WC_EXT_STEPS = 0, WC_EXT_BLOCKS = 1, WC_KMER = 2, WC_LF_STEPS = 3, WC_SA_READS = 4,
    WC_U_WALK = 5, WC_U_SAMPLE = 6, WC_U_TEXT = 7,   // U_*: extension of unique matches by text
    WC_JOINS = 8,                                     // locate: walks that stopped at a row of an earlier pass
    WC_JOIN_OFF = 9,                                  // locate: calls whose walked rows allowed no joins
    WC_N = 10
};
u64 *mb_work_counter_buf(cudaStream_t st);   // device array of WC_N u64 (zeroed on first use)

// Stage a host-or-device input on the device: returns a device pointer (the input itself when
// it already is one, else a copy in `buf`).
int mb_stage_in(const void *src, size_t bytes, cudaStream_t st, DevBuf &buf, const void **dev);

// ----------------------------------------------------------------------------- index layout
// One occurrence block per 64 BWT rows, 32 bytes: the counts of A, C, G, T in B[0, 64b) as four
// u32 (n < 2^32), then the 64 symbols of B[64b, 64b+64) as two bit planes: bit q of `lo` is the
// low bit of row q's 2-bit code, bit q of `hi` its high bit.  The $ row (primary) is stored as A
// and excluded from the counts.  The paper (Section 2.2) uses 64-byte blocks of 128 rows sized
// for a CPU cache line; on this GPU a random read costs one 32-byte DRAM sector, so a block is
// one sector and every LF step or block access reads exactly one.  The planes make the symbol of
// a row two bit tests and the count of a symbol before a row one 64-bit mask and popcount.
constexpr u32 BLK_SHIFT = 6;
constexpr u32 BLK_ROWS = 1u << BLK_SHIFT;
constexpr u32 BLK_MASK = BLK_ROWS - 1;
struct __align__(32) OccBlock {
    u32 cnt[4];
    u64 lo, hi;
};
static_assert(sizeof(OccBlock) == 32, "one block per 32-byte sector");

// Index view passed to kernels by value.
struct DevIndex {
    const OccBlock *occ;
    const u32 *ssa;     // S(x*r)
    const u32 *kmer;    // (k, kr, s) of every k-mer, base t of the k-mer in bits 2t..2t+1
    u64 n;              // |T|
    u64 primary;        // row with S = 0
    u64 C[4];           // C[a] = #{i : B[i] < a}, a = A,C,G,T
    u64 nblocks;
    u32 r;              // SA sample rate
    u32 kmer_k;
    const u32 *text2;   // T[0, n-1), 16 bases per word (null without the auxiliary arrays)
    const u32 *sa_aux;  // S(x * AUX_RATE)
    const u32 *isa_aux; // row of the suffix at text position p * AUX_RATE
};
// Sample rate of the auxiliary SA / ISA samples used to extend unique matches by comparison.
constexpr u32 AUX_RATE = 4;

struct mb_index_impl;

// ----------------------------------------------------------------------------- device helpers
// Every row, count and interval bound is below n < 2^32, so the kernels work in u32.
struct Blk {
    u32 c[4];
    u64 lo, hi;
};
// The whole block in one 256-bit load.
__device__ __forceinline__ Blk load_blk(const OccBlock *__restrict__ blk) {
    u64 c01, c23, lo, hi;
    asm("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(c01), "=l"(c23), "=l"(lo), "=l"(hi) : "l"(blk));
    Blk b;
    b.c[0] = (u32)c01; b.c[1] = (u32)(c01 >> 32); b.c[2] = (u32)c23; b.c[3] = (u32)(c23 >> 32);
    b.lo = lo; b.hi = hi;
    return b;
}

// Rows of the block before row m (0..63) as a bit mask.
__device__ __forceinline__ u64 rows_before(u32 m) { return (1ULL << m) - 1; }
// Code of row m of the block.
__device__ __forceinline__ u32 sym_at(const Blk &b, u32 m) {
    return (u32)((b.lo >> m) & 1) | ((u32)((b.hi >> m) & 1) << 1);
}
// Rows holding code a (0..3).
__device__ __forceinline__ u64 rows_eq(const Blk &b, u32 a) {
    const u64 fl = (u64)(a & 1) - 1, fh = (u64)(a >> 1) - 1;   // all ones where that bit of a is 0
    return (b.lo ^ fl) & (b.hi ^ fh);
}
// Rows holding a code <= a (0..3).
__device__ __forceinline__ u64 rows_le(const Blk &b, u32 a) {
    return a < 2 ? (a == 0 ? ~(b.lo | b.hi) : ~b.hi) : (a == 2 ? ~(b.lo & b.hi) : ~0ULL);
}
// #{rows before m holding code a}; the $ row (stored as A) is not corrected here.
__device__ __forceinline__ u32 cnt_sym(const Blk &b, u32 m, u32 a) { return __popcll(rows_eq(b, a) & rows_before(m)); }
// #{rows before m holding a code <= a}; the $ row (stored as A) is not corrected here.
__device__ __forceinline__ u32 cnt_le(const Blk &b, u32 m, u32 a) { return __popcll(rows_le(b, a) & rows_before(m)); }

// x[a] for a in 0..3 without dynamic indexing (which would go through local memory)
__device__ __forceinline__ u32 sel4(u32 a, u32 x0, u32 x1, u32 x2, u32 x3) {
    return a < 2 ? (a == 0 ? x0 : x1) : (a == 2 ? x2 : x3);
}

// [the $ row lies in the block of x, before x]
__device__ __forceinline__ u32 dollar_before(u32 x, u32 primary) {
    const u32 bstart = x & ~BLK_MASK;
    return (primary >= bstart && primary < x) ? 1u : 0u;
}

// One LF step of Algorithm 2 from row x (x is not the $ row): a = B[x], result C[a] + #a in
// B[0, x).
__device__ __forceinline__ u32 lf_blk(const Blk &b, u32 x, u32 primary, u32 C0, u32 C1, u32 C2, u32 C3) {
    const u32 m = x & BLK_MASK;
    const u32 a = sym_at(b, m);
    u32 cnt = cnt_sym(b, m, a);
    if (a == 0) cnt -= dollar_before(x, primary);
    return sel4(a, C0 + b.c[0], C1 + b.c[1], C2 + b.c[2], C3 + b.c[3]) + cnt;
}

// Algorithm 1 in one step.  Extends the interval (p, q, s) of P on the side of p by symbol a
// (0..3): p is lo of the strand being extended backwards, q is lo of the other strand.
//   s'  = #a in B[p, p+s)
//   p'  = C[a] + #a in B[0, p)
//   q'  = q + #{ $ or symbols > a } in B[p, p+s) = q + s - #{symbols <= a} in B[p, p+s)
// BackwardExt((k,k',s), a) is (p,q) = (k,k'); ForwardExt((k,k',s), a) is (p,q) = (k',k) with
// the complement of a.
struct Ext {
    u32 p, q, s;
};
// #a and #{symbols <= a} in B[0, x), $ excluded
__device__ __forceinline__ void occ_a_le(const Blk &b, u32 x, u32 a, u32 primary, u32 &na, u32 &nle) {
    const u32 m = x & BLK_MASK, d = dollar_before(x, primary);
    na = sel4(a, b.c[0], b.c[1], b.c[2], b.c[3]) + cnt_sym(b, m, a) - (a == 0 ? d : 0u);
    const u32 c01 = b.c[0] + b.c[1], c012 = c01 + b.c[2];
    nle = sel4(a, b.c[0], c01, c012, c012 + b.c[3]) + cnt_le(b, m, a) - d;
}

// One extension from the already loaded blocks b0 (of row p) and b1 (of row p+s).
__device__ __forceinline__ Ext extend_blocks(const DevIndex &I, const Blk &b0, const Blk &b1, u32 p, u32 q, u32 s,
                                             u32 a) {
    const u32 e = p + s, prim = (u32)I.primary;
    u32 na0, nle0, na1, nle1;
    occ_a_le(b0, p, a, prim, na0, nle0);
    occ_a_le(b1, e, a, prim, na1, nle1);
    Ext r;
    r.s = na1 - na0;
    r.p = sel4(a, (u32)I.C[0], (u32)I.C[1], (u32)I.C[2], (u32)I.C[3]) + na0;
    r.q = q + s - (nle1 - nle0);
    return r;
}

// One extension: the blocks of rows p and p+s are read once each (once in all when they are the
// same block).
__device__ __forceinline__ Ext extend(const DevIndex &I, u32 p, u32 q, u32 s, u32 a) {
    const u32 e = p + s;
    const Blk b0 = load_blk(I.occ + (p >> BLK_SHIFT));
    Blk b1 = b0;
    if ((e >> BLK_SHIFT) != (p >> BLK_SHIFT)) b1 = load_blk(I.occ + (e >> BLK_SHIFT));
    return extend_blocks(I, b0, b1, p, q, s, a);
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
// same size.  With n_dev (device), only the first min(n, *n_dev) items are sorted (an odd number
// of passes then still copies all n back).
struct BitRange {
    int lo, hi;
};
size_t radix_tmp_bytes(size_t n);
int radix_sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, size_t n, const BitRange *ranges,
                     int nranges, void *tmp, cudaStream_t st, const u64 *n_dev = nullptr);

// plan internals used by the server: device bytes of a plan, asynchronous copy of its result
// counts to host memory (3 u64: n_smem, n_hits, and the device error word in the upper half of
// the third), and its device result arrays
size_t mb_plan_bytes(const mb_plan *p);
// device bytes mb_plan_create would allocate for these limits (no allocation)
size_t mb_plan_workspace_bytes(const mb_opts *opts, u64 n, u32 max_reads, u64 max_bases, u64 max_smem,
                               u64 max_hits);
int mb_plan_counts_async(mb_plan *p, u64 *host_counts, cudaStream_t st);
void mb_plan_arrays(const mb_plan *p, const mb_smem **smem, const u32 **hits, u64 *max_smem, u64 *max_hits);
// seeding of a plan's batch without the locate (records with hit offsets), the plan's per-record
// known positions (NOPOS where seeding did not find one), and the locate of device records with
// such positions (hits at the records' offsets; every distinct row walked once)
int mb_plan_run_seed(mb_plan *p, const uint8_t *seq, const uint64_t *off, uint32_t n_reads, const uint8_t *mate,
                     cudaStream_t st);
const u32 *mb_plan_known(const mb_plan *p);
// SMEMs of reads already in device memory (what mb_seed_batch does after staging its inputs):
// read r is dseq[doff[r], doff[r+1]), o0 = doff[0] and o1 = doff[n_reads] as host values, dlc
// an optional per-read (l | c << 16); out may be host or device.  No pointer is classified
// except out.
int mb_seed_device(const mb_index *idx, const u8 *dseq, const u64 *doff, u32 n_reads, const u8 *dmate,
                   const u32 *dlc, u64 o0, u64 o1, const mb_opts *opts, cudaStream_t st, mb_smem *out, u64 cap,
                   u64 *n_out, u64 *n_hits);
// Locate of device records (their hits at their hit offsets), D walks per lane, walks that join
// when `join`, walks to the rate-4 samples when `aux`; workspace allocated in stream order.
int mb_locate_records(const mb_index *idx, const mb_smem *sm, u64 n_smem, const u32 *known, u32 *hits, u64 n_hits,
                      u32 depth, bool join, bool aux, cudaStream_t st);
// build flags of an index (MB_BS3 for the 3-base bisulfite index)
u32 mb_index_flags(const mb_index *x);
// drops the host-buffer pipelines kept for an index (called when the index is freed)
void mb_pipeline_forget(const mb_index *idx);

inline unsigned grid_for(size_t n, unsigned block, unsigned cap = 152u * 64u) {
    size_t g = (n + block - 1) / block;
    if (g > cap) g = cap;
    if (g == 0) g = 1;
    return (unsigned)g;
}
