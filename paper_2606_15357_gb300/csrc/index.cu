// FMD-index construction on the GPU (Section 2.1 definitions, Section 2.2 block layout (here one
// 32-byte block per 64 rows),
// Section 2.4 sampled suffix array, Section 2.5 k-mer ds-interval table).
//
//   T = R . revcomp(R) . $            (bisulfite: R -> CT(R) . GA(R), Section 2.9)
//   S = suffix array of T             prefix doubling: sort by the first 27 symbols, then
//                                     repeatedly re-sort the suffixes whose 2h-prefix is still
//                                     shared by (rank of the h-prefix, rank of the h-prefix at +h)
//   B[i] = T[S(i) - 1], T[-1] = $     written straight into 32-byte occurrence blocks
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include "common.cuh"

struct mb_index {
    u64 n = 0, rlen = 0, primary = 0;
    u32 sa_rate = 32, kmer_k = 10, flags = 0;
    u64 C[5] = {0, 0, 0, 0, 0};   // $, A, C, G, T
    u64 nblocks = 0;
    OccBlock *occ = nullptr;
    u32 *ssa = nullptr;
    u32 *kmer = nullptr;
    u32 *sa = nullptr;            // full SA, kept until mb_index_drop_sa
    // for extending unique matches by text comparison (absent with MB_NO_AUX)
    u32 *text2 = nullptr;         // T[0, n-1) at 2 bits per base, 16 per word, first in the low bits
    u32 *sa_aux = nullptr;        // S(x * AUX_RATE)
    u32 *isa_aux = nullptr;       // row of the suffix at text position p * AUX_RATE
    int device = 0;
};

u64 text2_words(u64 n) { return (n - 1 + 15) / 16 + 2; }   // two words of padding for unaligned reads
u64 aux_count(u64 n) { return (n + AUX_RATE - 1) / AUX_RATE; }

DevIndex mb_dev_index(const mb_index *x) {
    DevIndex I;
    I.occ = x->occ;
    I.ssa = x->ssa;
    I.kmer = x->kmer;
    I.n = x->n;
    I.primary = x->primary;
    for (int a = 0; a < 4; ++a) I.C[a] = x->C[a + 1];
    I.nblocks = x->nblocks;
    I.r = x->sa_rate;
    I.kmer_k = x->kmer_k;
    I.text2 = x->text2;
    I.sa_aux = x->sa_aux;
    I.isa_aux = x->isa_aux;
    return I;
}
int mb_index_device(const mb_index *x) { return x->device; }
u32 mb_index_flags(const mb_index *x) { return x->flags; }

namespace {

constexpr u64 GOLDEN = 0x9E3779B97F4A7C15ULL;
constexpr int KEY_SYMS = 27;   // 5^27 < 2^63: the first 27 symbols of a suffix in base 5 ($ = 0)

__device__ __forceinline__ u8 ref_base(const u8 *__restrict__ R, u64 x, u64 seed) {
    u8 b = R[x];
    return b < 4 ? b : (u8)(mb_mix64(seed + (x + 1) * GOLDEN) >> 62);
}
__device__ __forceinline__ u8 r3_base(const u8 *__restrict__ R, u64 m, u64 x, u64 seed, int bs3) {
    if (!bs3) return ref_base(R, x, seed);
    if (x < m) {
        u8 b = ref_base(R, x, seed);
        return b == 1 ? 3 : b;   // C -> T
    }
    u8 b = ref_base(R, x - m, seed);
    return b == 2 ? 0 : b;       // G -> A
}

// T[i] in 0..3 for i < n-1; T[n-1] = 4 marks $.
__global__ void k_pack_text(const u8 *__restrict__ R, u64 m, u64 seed, int bs3, u8 *__restrict__ T, u64 n) {
    const u64 M = (n - 1) / 2;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        u8 b;
        if (i == n - 1) b = 4;
        else if (i < M) b = r3_base(R, m, i, seed, bs3);
        else b = (u8)(3 - r3_base(R, m, 2 * M - 1 - i, seed, bs3));
        T[i] = b;
    }
}

__global__ void k_init_keys(const u8 *__restrict__ T, u64 n, u64 *__restrict__ keys, u32 *__restrict__ vals) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        u64 v = 0;
#pragma unroll
        for (int q = 0; q < KEY_SYMS; ++q) {
            u64 p = i + q;
            u32 s = p < n - 1 ? (u32)T[p] + 1u : 0u;
            v = v * 5 + s;
        }
        keys[i] = v;
        vals[i] = (u32)i;
    }
}

// hv[t] = (start of a new key run) ? pos(t) : 0, for a max-scan giving each item its run head.
// flag[t] = item t is in a run of more than one key.
__global__ void k_heads(const u64 *__restrict__ keys, const u32 *__restrict__ pos, u64 A, u32 *__restrict__ hv,
                        u32 *__restrict__ flag) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < A; t += (u64)gridDim.x * blockDim.x) {
        u64 k = keys[t];
        bool head = t == 0 || keys[t - 1] != k;
        bool last = t == A - 1 || keys[t + 1] != k;
        hv[t] = head ? (pos ? pos[t] : (u32)t) : 0u;
        flag[t] = (head && last) ? 0u : 1u;
    }
}

__global__ void k_set_rank(const u32 *__restrict__ sa_vals, const u32 *__restrict__ hv, u64 A, u32 *__restrict__ rank) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < A; t += (u64)gridDim.x * blockDim.x)
        rank[sa_vals[t]] = hv[t];
}

// act2[pos[t]] = (act ? act[t] : t) for flagged t
__global__ void k_compact(const u32 *__restrict__ flag, const u32 *__restrict__ pos, const u32 *__restrict__ act,
                          u64 A, u32 *__restrict__ act2) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < A; t += (u64)gridDim.x * blockDim.x)
        if (flag[t]) act2[pos[t]] = act ? act[t] : (u32)t;
}

__global__ void k_round_keys(const u32 *__restrict__ act, u64 A, const u32 *__restrict__ SA,
                             const u32 *__restrict__ rank, u64 h, u64 n, u64 *__restrict__ keys,
                             u32 *__restrict__ vals, u32 *__restrict__ err) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < A; t += (u64)gridDim.x * blockDim.x) {
        u32 p = SA[act[t]];
        u64 q = (u64)p + h;
        u32 r2 = 0;
        if (q < n) r2 = rank[q];
        else atomicOr(err, 1u);   // a suffix whose h-prefix holds $ is unique; never active
        keys[t] = ((u64)rank[p] << 32) | r2;
        vals[t] = p;
    }
}

__global__ void k_scatter_sa(const u32 *__restrict__ act, u64 A, const u32 *__restrict__ vals, u32 *__restrict__ SA) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < A; t += (u64)gridDim.x * blockDim.x)
        SA[act[t]] = vals[t];
}

// One warp per 128 rows, i.e. two 64-row blocks: symbols B[x] = T[S(x)-1] packed 2 bits each
// ($ stored as A), per-block counts of A,C,G,T (excluding $) to bcnt[a * nblocks + b].
__global__ void k_bwt_blocks(const u8 *__restrict__ T, const u32 *__restrict__ SA, u64 n, OccBlock *__restrict__ occ,
                             u64 nblocks, u64 *__restrict__ bcnt, u64 *__restrict__ primary) {
    const int lane = threadIdx.x & 31;
    const u64 warps = (u64)gridDim.x * (blockDim.x >> 5);
    const u64 ngroups = (nblocks + 1) / 2;
    for (u64 g = blockIdx.x * (u64)(blockDim.x >> 5) + (threadIdx.x >> 5); g < ngroups; g += warps) {
        u32 lob = 0, hib = 0, c[4] = {0, 0, 0, 0};   // low / high code bits of the lane's 4 rows
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            u64 x = g * 128 + (u64)lane * 4 + j;
            if (x < n) {
                u32 p = SA[x];
                u32 s;
                if (p == 0) {
                    *primary = x;
                    s = 0;
                } else {
                    s = T[p - 1];
                    c[s] += 1;
                }
                lob |= (s & 1u) << j;
                hib |= (s >> 1) << j;
            }
        }
        // rows 4*(lane & 15) .. +3 of block 2g + (lane >> 4): OR the planes over each 16-lane half
        u64 lo = (u64)lob << (4 * (lane & 15)), hi = (u64)hib << (4 * (lane & 15));
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
            lo |= __shfl_xor_sync(0xffffffffu, lo, d);
            hi |= __shfl_xor_sync(0xffffffffu, hi, d);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int d = 8; d > 0; d >>= 1) c[a] += __shfl_xor_sync(0xffffffffu, c[a], d);   // per 16-lane half
        const u64 b = 2 * g + (u64)(lane >> 4);
        if (b < nblocks) {
            if ((lane & 15) == 0) {
                occ[b].lo = lo;
                occ[b].hi = hi;
            }
            const u32 a = (u32)(lane & 15);
            if (a < 4) bcnt[(u64)a * nblocks + b] = a < 2 ? (a == 0 ? c[0] : c[1]) : (a == 2 ? c[2] : c[3]);
        }
    }
}

__global__ void k_fill_counts(const u64 *__restrict__ bcnt_scanned, u64 nblocks, OccBlock *__restrict__ occ) {
    for (u64 b = blockIdx.x * (u64)blockDim.x + threadIdx.x; b < nblocks; b += (u64)gridDim.x * blockDim.x)
#pragma unroll
        for (int a = 0; a < 4; ++a) occ[b].cnt[a] = (u32)bcnt_scanned[(u64)a * nblocks + b];
}

__global__ void k_sample_sa(const u32 *__restrict__ SA, u64 n, u32 r, u32 *__restrict__ ssa) {
    u64 m = (n + r - 1) / r;
    for (u64 x = blockIdx.x * (u64)blockDim.x + threadIdx.x; x < m; x += (u64)gridDim.x * blockDim.x)
        ssa[x] = SA[x * r];
}

// T[0, n-1) packed 16 bases per u32 word, base e of word w at bits 2e..2e+1; padding words zero.
__global__ void k_text2(const u8 *__restrict__ T, u64 n, u32 *__restrict__ t2, u64 words) {
    for (u64 w = blockIdx.x * (u64)blockDim.x + threadIdx.x; w < words; w += (u64)gridDim.x * blockDim.x) {
        u32 v = 0;
        for (u32 e = 0; e < 16; ++e) {
            const u64 x = 16 * w + e;
            if (x < n - 1) v |= (u32)(T[x] & 3u) << (2 * e);
        }
        t2[w] = v;
    }
}

// isa[p / r] = the row of the suffix at text position p, for p a multiple of r
__global__ void k_sample_isa(const u32 *__restrict__ SA, u64 n, u32 r, u32 *__restrict__ isa) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const u32 p = SA[i];
        if (p % r == 0) isa[p / r] = (u32)i;
    }
}

// ds-interval of every k-mer by k BackwardExt steps from the empty string (0, 0, n).  The
// k-mer of entry w has its t-th base (t = 0 first) in bits 2t..2t+1 of w.
__global__ void k_kmer_table(DevIndex I, u32 k, u32 *__restrict__ out) {
    u64 nk = 1ULL << (2 * k);
    for (u64 w = blockIdx.x * (u64)blockDim.x + threadIdx.x; w < nk; w += (u64)gridDim.x * blockDim.x) {
        u32 p = 0, q = 0, s = (u32)I.n;
        for (int t = (int)k - 1; t >= 0; --t) {
            u32 a = (u32)(w >> (2 * t)) & 3u;
            Ext e = extend(I, p, q, s, a);
            p = e.p; q = e.q; s = e.s;
        }
        out[3 * w + 0] = p;
        out[3 * w + 1] = q;
        out[3 * w + 2] = s;
    }
}

int nbits(u64 v) {   // smallest b with v <= 2^b
    int b = 0;
    while (b < 64 && (1ULL << b) < v) ++b;
    return b;
}

}  // namespace

// ============================================================================ host side
static std::mutex g_err_mu;
static std::string g_err;
void mb_set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> g(g_err_mu);
    g_err = buf;
}
extern "C" const char *mb_last_error(void) {
    static thread_local std::string copy;
    std::lock_guard<std::mutex> g(g_err_mu);
    copy = g_err;
    return copy.c_str();
}

// ----------------------------------------------------------------------------- measurement hooks
static std::atomic<u64> g_launches{0};
static std::atomic<int> g_prof{0};
struct KStat {
    double ms = 0;
    u64 launches = 0;
};
static std::map<std::string, KStat> g_kstat;
void mb_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

KTimer::KTimer(const char *n, cudaStream_t s) : name(n), st(s) {
    if (g_prof.load()) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
}
void KTimer::start() {
    if (a) cudaEventRecord(a, st);
}
void KTimer::stop() {
    if (b) cudaEventRecord(b, st);
}
KTimer::~KTimer() {
    if (!a) return;
    float ms = 0;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
        std::lock_guard<std::mutex> g(g_err_mu);
        KStat &k = g_kstat[name];
        k.ms += ms;
        k.launches += 1;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
}

static u64 *g_wc = nullptr;
static int g_wc_dev = -1;
u64 *mb_work_counter_buf(cudaStream_t st) {
    int d = 0;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> g(g_err_mu);
    if (!g_wc || g_wc_dev != d) {
        if (cudaMalloc(&g_wc, WC_N * sizeof(u64)) != cudaSuccess) return nullptr;
        cudaMemsetAsync(g_wc, 0, WC_N * sizeof(u64), st);
        g_wc_dev = d;
    }
    return g_wc;
}

extern "C" void mb_profile_enable(int on) { g_prof.store(on ? 1 : 0); }
extern "C" int mb_profile_get(const char *kernel, double *ms, uint64_t *launches) {
    if (!kernel) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(g_err_mu);
    auto it = g_kstat.find(kernel);
    if (ms) *ms = it == g_kstat.end() ? 0.0 : it->second.ms;
    if (launches) *launches = it == g_kstat.end() ? 0 : it->second.launches;
    return MB_OK;
}
extern "C" void mb_profile_reset(void) {
    {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_kstat.clear();
    }
    if (g_wc) {
        cudaDeviceSynchronize();
        cudaMemset(g_wc, 0, WC_N * sizeof(u64));
    }
}
extern "C" uint64_t mb_launch_count(void) { return g_launches.load(); }
extern "C" void mb_work_counters_all(uint64_t *out, uint32_t count) {
    u64 v[WC_N] = {};
    if (g_wc) {
        cudaDeviceSynchronize();
        cudaMemcpy(v, g_wc, sizeof v, cudaMemcpyDeviceToHost);
    }
    for (u32 i = 0; i < count; ++i) out[i] = i < (u32)WC_N ? v[i] : 0;
}

extern "C" void mb_work_counters(uint64_t *ext_steps, uint64_t *ext_blocks, uint64_t *kmer_lookups,
                                 uint64_t *lf_steps, uint64_t *sa_reads) {
    u64 v[WC_N] = {};
    if (g_wc) {
        cudaDeviceSynchronize();
        cudaMemcpy(v, g_wc, sizeof v, cudaMemcpyDeviceToHost);
    }
    if (ext_steps) *ext_steps = v[WC_EXT_STEPS];
    if (ext_blocks) *ext_blocks = v[WC_EXT_BLOCKS];
    if (kmer_lookups) *kmer_lookups = v[WC_KMER];
    if (lf_steps) *lf_steps = v[WC_LF_STEPS];
    if (sa_reads) *sa_reads = v[WC_SA_READS];
}

void mb_keep_pool_memory() {
    static thread_local int done_dev = -1;
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d == done_dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
        u64 thr = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done_dev = d;
}

bool mb_is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device allocation holding p, from the driver's cuMemGetAddressRange (looked up once through
// the runtime's driver entry points, so the library does not link the driver directly).
static bool device_range(const void *p, u64 *base, u64 *size) {
    typedef int (*AddrRange)(unsigned long long *, size_t *, unsigned long long);
    static AddrRange fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (AddrRange)f;
        cudaGetLastError();
    });
    if (!fn) return false;
    unsigned long long b = 0;
    size_t z = 0;
    if (fn(&b, &z, (unsigned long long)(uintptr_t)p) != 0) return false;
    *base = b;
    *size = z;
    return true;
}

extern "C" int mb_device_extent(const void *p, uint64_t *base, uint64_t *size) {
    if (!p || !base || !size || !mb_is_device_ptr(p)) return MB_ERR_ARG;
    u64 b = 0, z = 0;
    if (!device_range(p, &b, &z)) {
        mb_set_error("mb_device_extent: the driver does not report the allocation of %p", p);
        return MB_ERR_CUDA;
    }
    *base = b;
    *size = z;
    return MB_OK;
}

int mb_check_span(const void *p, u64 bytes, const char *what) {
    if (!p || bytes == 0 || !mb_is_device_ptr(p)) return MB_OK;
    u64 b = 0, z = 0;
    if (!device_range(p, &b, &z)) return MB_OK;   // the driver cannot tell: nothing to check
    const u64 a = (u64)(uintptr_t)p;
    if (a < b || a - b > z || bytes > z - (a - b)) {
        mb_set_error("%s: %llu bytes from %p pass the end of its device allocation (%llu bytes from 0x%llx)", what,
                     (unsigned long long)bytes, p, (unsigned long long)z, (unsigned long long)b);
        return MB_ERR_ARG;
    }
    return MB_OK;
}

int mb_stage_in(const void *src, size_t bytes, cudaStream_t st, DevBuf &buf, const void **dev) {
    if (bytes == 0 || mb_is_device_ptr(src)) {
        *dev = src;
        return MB_OK;
    }
    MB_TRY(buf.alloc(bytes, st));
    MB_CK(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = buf.p;
    return MB_OK;
}

static void free_index(mb_index *x) {
    if (!x) return;
    if (x->occ) cudaFree(x->occ);
    if (x->ssa) cudaFree(x->ssa);
    if (x->kmer) cudaFree(x->kmer);
    if (x->sa) cudaFree(x->sa);
    if (x->text2) cudaFree(x->text2);
    if (x->sa_aux) cudaFree(x->sa_aux);
    if (x->isa_aux) cudaFree(x->isa_aux);
    delete x;
}

// Suffix array of T (device, n symbols) by prefix doubling.  SA (device, n) receives it.
static int build_sa(const u8 *T, u64 n, u32 *SA, cudaStream_t st) {
    // 25 bytes per suffix: keys and the sort's spare keys (8 + 8), values and spare values (4 + 4),
    // ranks (4), two active lists (4 + 4); the run heads and flags (4 + 4) live in the spare keys,
    // which are free whenever they are used.
    DevBuf bk, bka, bv, bva, btmp, brank, bact, bact2, berr, bcount;
    MB_TRY(bk.alloc(n * 8, st));
    MB_TRY(bka.alloc(n * 8, st));
    MB_TRY(bv.alloc(n * 4, st));
    MB_TRY(bva.alloc(n * 4, st));
    size_t tb = radix_tmp_bytes(n);
    size_t sb = scan_tmp_bytes(n);
    MB_TRY(btmp.alloc(tb > sb ? tb : sb, st));
    MB_TRY(brank.alloc(n * 4, st));
    MB_TRY(bact.alloc(n * 4, st));
    MB_TRY(bact2.alloc(n * 4, st));
    MB_TRY(berr.alloc(8, st));
    MB_TRY(bcount.alloc(8, st));
    u64 *keys = bk.as<u64>(), *keys_alt = bka.as<u64>();
    u32 *vals = bv.as<u32>(), *vals_alt = bva.as<u32>();
    u32 *rank = brank.as<u32>(), *hv = bka.as<u32>(), *flag = bka.as<u32>() + n;
    u32 *act = bact.as<u32>(), *act2 = bact2.as<u32>();
    u32 *err = berr.as<u32>(), *count = bcount.as<u32>();
    MB_CK(cudaMemsetAsync(err, 0, 4, st));
    const unsigned B = 256;

    // round 0: the first 27 symbols
    k_init_keys<<<grid_for(n, B), B, 0, st>>>(T, n, keys, vals);
    MB_KCHECK();
    BitRange r0[1] = {{0, 63}};
    MB_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, r0, 1, btmp.p, st));
    MB_CK(cudaMemcpyAsync(SA, vals, n * 4, cudaMemcpyDeviceToDevice, st));
    k_heads<<<grid_for(n, B), B, 0, st>>>(keys, nullptr, n, hv, flag);
    MB_KCHECK();
    MB_TRY(scan_inclusive_max_u32(hv, hv, n, btmp.p, st));
    k_set_rank<<<grid_for(n, B), B, 0, st>>>(vals, hv, n, rank);
    MB_KCHECK();
    MB_TRY(scan_exclusive_u32(flag, hv, n, count, btmp.p, st));   // hv reused as positions
    k_compact<<<grid_for(n, B), B, 0, st>>>(flag, hv, nullptr, n, act);
    MB_KCHECK();
    u32 A = 0;
    MB_CK(cudaMemcpyAsync(&A, count, 4, cudaMemcpyDeviceToHost, st));
    MB_CK(cudaStreamSynchronize(st));

    const int nb = nbits(n);
    BitRange rr[2] = {{0, nb}, {32, 32 + nb}};
    u64 h = KEY_SYMS;
    while (A > 0) {
        k_round_keys<<<grid_for(A, B), B, 0, st>>>(act, A, SA, rank, h, n, keys, vals, err);
        MB_KCHECK();
        MB_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, A, rr, 2, btmp.p, st));
        k_scatter_sa<<<grid_for(A, B), B, 0, st>>>(act, A, vals, SA);
        MB_KCHECK();
        k_heads<<<grid_for(A, B), B, 0, st>>>(keys, act, A, hv, flag);
        MB_KCHECK();
        MB_TRY(scan_inclusive_max_u32(hv, hv, A, btmp.p, st));
        k_set_rank<<<grid_for(A, B), B, 0, st>>>(vals, hv, A, rank);
        MB_KCHECK();
        MB_TRY(scan_exclusive_u32(flag, hv, A, count, btmp.p, st));
        k_compact<<<grid_for(A, B), B, 0, st>>>(flag, hv, act, A, act2);
        MB_KCHECK();
        u32 A2 = 0, e = 0;
        MB_CK(cudaMemcpyAsync(&A2, count, 4, cudaMemcpyDeviceToHost, st));
        MB_CK(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, st));
        MB_CK(cudaStreamSynchronize(st));
        if (e) {
            mb_set_error("suffix sort: an active suffix reached past the end of T (h=%llu)",
                         (unsigned long long)h);
            return MB_ERR_DEVICE_CHECK;
        }
        u32 *t = act; act = act2; act2 = t;
        A = A2;
        h *= 2;
        if (h > 2 * n + 64) {
            mb_set_error("suffix sort did not converge");
            return MB_ERR_DEVICE_CHECK;
        }
    }
    return MB_OK;
}

extern "C" int mb_index_build(const uint8_t *ref, uint64_t len, const mb_opts *opts, uint64_t n_seed,
                              void *stream, mb_index **out) {
    if (!ref || !out || len == 0) {
        mb_set_error("mb_index_build: null argument or empty reference");
        return MB_ERR_ARG;
    }
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    u32 flags = opts ? opts->flags : 0;
    u32 r = opts && opts->sa_rate ? opts->sa_rate : 32;
    u32 kk = opts && opts->kmer_k ? opts->kmer_k : 10;
    if (kk > 16 || r == 0) {
        mb_set_error("mb_index_build: kmer_k must be <= 16 and sa_rate > 0");
        return MB_ERR_ARG;
    }
    int bs3 = (flags & MB_BS3) ? 1 : 0;
    u64 M = bs3 ? 2 * len : len;
    u64 n = 2 * M + 1;
    if (n >= (1ULL << 32)) {
        mb_set_error("mb_index_build: n = %llu must be below 2^32", (unsigned long long)n);
        return MB_ERR_ARG;
    }
    mb_index *X = new mb_index;
    X->n = n;
    X->rlen = M;
    X->sa_rate = r;
    X->kmer_k = kk;
    X->flags = flags & MB_BS3;
    cudaGetDevice(&X->device);
    int rc = MB_OK;
    do {
        DevBuf bref, bT, bcnt, btmp, bprim, btot;
        const void *dref = nullptr;
        if ((rc = mb_stage_in(ref, len, st, bref, &dref)) != MB_OK) break;
        if ((rc = bT.alloc(n, st)) != MB_OK) break;
        k_pack_text<<<grid_for(n, 256), 256, 0, st>>>((const u8 *)dref, len, n_seed, bs3, bT.as<u8>(), n);
        if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        bref.release();
        if (cudaMalloc(&X->sa, n * 4) != cudaSuccess) { rc = MB_ERR_NOMEM; break; }
        if ((rc = build_sa(bT.as<u8>(), n, X->sa, st)) != MB_OK) break;

        // BWT in occurrence blocks
        X->nblocks = n / BLK_ROWS + 1;
        const u64 nbk = X->nblocks;
        if (cudaMalloc(&X->occ, nbk * sizeof(OccBlock)) != cudaSuccess) { rc = MB_ERR_NOMEM; break; }
        if (cudaMemsetAsync(X->occ, 0, nbk * sizeof(OccBlock), st) != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        if ((rc = bcnt.alloc(nbk * 4 * 8, st)) != MB_OK) break;
        if ((rc = btmp.alloc(scan_tmp_bytes(nbk), st)) != MB_OK) break;
        if ((rc = bprim.alloc(8, st)) != MB_OK) break;
        if ((rc = btot.alloc(4 * 8, st)) != MB_OK) break;
        k_bwt_blocks<<<grid_for((nbk + 1) / 2 * 32, 256), 256, 0, st>>>(bT.as<u8>(), X->sa, n, X->occ, nbk, bcnt.as<u64>(),
                                                              bprim.as<u64>());
        if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        for (int a = 0; a < 4 && rc == MB_OK; ++a)
            rc = scan_exclusive_u64(bcnt.as<u64>() + a * nbk, bcnt.as<u64>() + a * nbk, nbk, btot.as<u64>() + a,
                                    btmp.p, st);
        if (rc != MB_OK) break;
        k_fill_counts<<<grid_for(nbk, 256), 256, 0, st>>>(bcnt.as<u64>(), nbk, X->occ);
        if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        u64 tot[4], prim = 0;
        if (cudaMemcpyAsync(tot, btot.p, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&prim, bprim.p, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        X->primary = prim;
        X->C[0] = 0;
        X->C[1] = 1;
        for (int a = 1; a < 4; ++a) X->C[a + 1] = X->C[a] + tot[a - 1];

        // sampled SA and k-mer table
        u64 ns = (n + r - 1) / r;
        if (cudaMalloc(&X->ssa, ns * 4) != cudaSuccess) { rc = MB_ERR_NOMEM; break; }
        k_sample_sa<<<grid_for(ns, 256), 256, 0, st>>>(X->sa, n, r, X->ssa);
        if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        u64 nk = 1ULL << (2 * kk);
        if (cudaMalloc(&X->kmer, nk * 12) != cudaSuccess) { rc = MB_ERR_NOMEM; break; }
        k_kmer_table<<<grid_for(nk, 256), 256, 0, st>>>(mb_dev_index(X), kk, X->kmer);
        if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        if (!(flags & MB_NO_AUX)) {
            // packed text and dense SA / ISA samples for extending unique matches by comparison
            const u64 tw = text2_words(n), na = aux_count(n);
            if (cudaMalloc(&X->text2, tw * 4) != cudaSuccess || cudaMalloc(&X->sa_aux, na * 4) != cudaSuccess ||
                cudaMalloc(&X->isa_aux, na * 4) != cudaSuccess) { rc = MB_ERR_NOMEM; break; }
            k_text2<<<grid_for(tw, 256), 256, 0, st>>>(bT.as<u8>(), n, X->text2, tw);
            k_sample_sa<<<grid_for(na, 256), 256, 0, st>>>(X->sa, n, AUX_RATE, X->sa_aux);
            k_sample_isa<<<grid_for(n, 256), 256, 0, st>>>(X->sa, n, AUX_RATE, X->isa_aux);
            if (cudaGetLastError() != cudaSuccess) { rc = MB_ERR_CUDA; break; }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MB_ERR_CUDA; break; }
    } while (0);
    {
        // give the build's temporaries (tens of GB at 1 Gbp) back to the device
        cudaStreamSynchronize(st);
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
        cudaGetLastError();
    }
    if (rc != MB_OK) {
        cudaStreamSynchronize(st);
        free_index(X);
        return rc;
    }
    *out = X;
    return MB_OK;
}

extern "C" void mb_index_free(mb_index *idx) {
    mb_pipeline_forget(idx);
    free_index(idx);
}

extern "C" int mb_index_info(const mb_index *idx, uint64_t *n, uint64_t *primary, uint64_t *ref_len) {
    if (!idx) return MB_ERR_ARG;
    if (n) *n = idx->n;
    if (primary) *primary = idx->primary;
    if (ref_len) *ref_len = idx->rlen;
    return MB_OK;
}

extern "C" int mb_index_drop_sa(mb_index *idx) {
    if (!idx) return MB_ERR_ARG;
    if (idx->sa) cudaFree(idx->sa);
    idx->sa = nullptr;
    return MB_OK;
}

static int copy_out(void *dst, const void *src, size_t bytes) {
    if (!dst || bytes == 0) return MB_OK;
    MB_CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
    return MB_OK;
}

namespace {
__global__ void k_kmer_get(const u32 *__restrict__ kmer, const u64 *__restrict__ codes, u64 n, u32 *__restrict__ out) {
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        const u64 w = codes[i];
        out[3 * i + 0] = kmer[3 * w + 0];
        out[3 * i + 1] = kmer[3 * w + 1];
        out[3 * i + 2] = kmer[3 * w + 2];
    }
}
}  // namespace

extern "C" int mb_index_kmer_get(const mb_index *idx, const uint64_t *codes, uint64_t n, uint32_t *out) {
    if (!idx || !idx->kmer || (n && (!codes || !out))) {
        mb_set_error("mb_index_kmer_get: null argument");
        return MB_ERR_ARG;
    }
    const u64 nk = 1ULL << (2 * idx->kmer_k);
    for (u64 i = 0; i < n; ++i)
        if (codes[i] >= nk) {
            mb_set_error("mb_index_kmer_get: code %llu is not below 4^%u", (unsigned long long)codes[i], idx->kmer_k);
            return MB_ERR_ARG;
        }
    if (n == 0) return MB_OK;
    DevBuf dc, dout;
    MB_TRY(dc.alloc(n * 8, 0));
    MB_TRY(dout.alloc(n * 12, 0));
    MB_CK(cudaMemcpy(dc.p, codes, n * 8, cudaMemcpyHostToDevice));
    k_kmer_get<<<grid_for(n, 256), 256>>>(idx->kmer, dc.as<u64>(), n, dout.as<u32>());
    MB_KCHECK();
    MB_CK(cudaMemcpy(out, dout.p, n * 12, cudaMemcpyDeviceToHost));
    return MB_OK;
}

extern "C" int mb_index_export(const mb_index *idx, uint32_t *sa, uint8_t *bwt, uint32_t *ssa, void *occ_blocks,
                               uint32_t *kmer, uint64_t *C) {
    if (!idx) return MB_ERR_ARG;
    if ((sa || bwt) && !idx->sa) {
        mb_set_error("mb_index_export: the full suffix array was dropped");
        return MB_ERR_ARG;
    }
    MB_TRY(copy_out(sa, idx->sa, idx->n * 4));
    if (bwt) {
        // decode B from the blocks on the host side of the caller's buffer
        std::vector<OccBlock> blk(idx->nblocks);
        MB_CK(cudaMemcpy(blk.data(), idx->occ, idx->nblocks * sizeof(OccBlock), cudaMemcpyDeviceToHost));
        std::vector<u8> b(idx->n);
        for (u64 x = 0; x < idx->n; ++x) {
            const OccBlock &o = blk[x >> BLK_SHIFT];
            const u32 m = (u32)(x & BLK_MASK);
            b[x] = x == idx->primary ? 0 : (u8)((((o.lo >> m) & 1) | (((o.hi >> m) & 1) << 1)) + 1);
        }
        MB_TRY(copy_out(bwt, b.data(), idx->n));
    }
    MB_TRY(copy_out(ssa, idx->ssa, ((idx->n + idx->sa_rate - 1) / idx->sa_rate) * 4));
    MB_TRY(copy_out(occ_blocks, idx->occ, idx->nblocks * sizeof(OccBlock)));
    MB_TRY(copy_out(kmer, idx->kmer, (1ULL << (2 * idx->kmer_k)) * 12));
    if (C) memcpy(C, idx->C, sizeof(idx->C));
    return MB_OK;
}

extern "C" int mb_index_export_aux(const mb_index *idx, uint32_t *text2, uint32_t *sa_aux, uint32_t *isa_aux) {
    if (!idx) return MB_ERR_ARG;
    if (!idx->text2 && (text2 || sa_aux || isa_aux)) {
        mb_set_error("mb_index_export_aux: the index was built without the auxiliary arrays");
        return MB_ERR_ARG;
    }
    if (!idx->text2) return MB_OK;
    MB_TRY(copy_out(text2, idx->text2, text2_words(idx->n) * 4));
    MB_TRY(copy_out(sa_aux, idx->sa_aux, aux_count(idx->n) * 4));
    MB_TRY(copy_out(isa_aux, idx->isa_aux, aux_count(idx->n) * 4));
    return MB_OK;
}

// ----------------------------------------------------------------------------- save / load
namespace {
constexpr u64 MAGIC = 0x3130585744424D4DULL;   // "MMBDWX01"
struct FileHeader {
    u64 magic, version, n, rlen, primary, nblocks;
    u32 sa_rate, kmer_k, flags, aux;   // aux: the SA / ISA sample rate when the packed text and
                                       // those samples follow, else 0
    u64 C[5];
    u64 checksum;
};
u64 checksum_words(const void *p, size_t bytes, u64 h) {
    const u8 *b = (const u8 *)p;
    size_t nw = bytes / 8;
    for (size_t i = 0; i < nw; ++i) {
        u64 w;
        memcpy(&w, b + 8 * i, 8);
        h = (h ^ w) * 0x100000001B3ULL;
        h ^= h >> 29;
    }
    for (size_t i = nw * 8; i < bytes; ++i) h = (h ^ b[i]) * 0x100000001B3ULL;
    return h;
}
}  // namespace

extern "C" int mb_index_save(const mb_index *idx, const char *path) {
    if (!idx || !path) return MB_ERR_ARG;
    u64 ns = (idx->n + idx->sa_rate - 1) / idx->sa_rate, nk = 1ULL << (2 * idx->kmer_k);
    const bool aux = idx->text2 != nullptr;
    std::vector<u8> occ(idx->nblocks * sizeof(OccBlock)), ssa(ns * 4), km(nk * 12);
    std::vector<u8> t2(aux ? text2_words(idx->n) * 4 : 0), sx(aux ? aux_count(idx->n) * 4 : 0), ix(sx.size());
    MB_CK(cudaMemcpy(occ.data(), idx->occ, occ.size(), cudaMemcpyDeviceToHost));
    MB_CK(cudaMemcpy(ssa.data(), idx->ssa, ssa.size(), cudaMemcpyDeviceToHost));
    MB_CK(cudaMemcpy(km.data(), idx->kmer, km.size(), cudaMemcpyDeviceToHost));
    if (aux) {
        MB_CK(cudaMemcpy(t2.data(), idx->text2, t2.size(), cudaMemcpyDeviceToHost));
        MB_CK(cudaMemcpy(sx.data(), idx->sa_aux, sx.size(), cudaMemcpyDeviceToHost));
        MB_CK(cudaMemcpy(ix.data(), idx->isa_aux, ix.size(), cudaMemcpyDeviceToHost));
    }
    std::vector<u8> *sec[] = {&occ, &ssa, &km, &t2, &sx, &ix};
    FileHeader h;
    memset(&h, 0, sizeof h);
    h.magic = MAGIC;
    h.version = 4;
    h.aux = aux ? AUX_RATE : 0u;
    h.n = idx->n;
    h.rlen = idx->rlen;
    h.primary = idx->primary;
    h.nblocks = idx->nblocks;
    h.sa_rate = idx->sa_rate;
    h.kmer_k = idx->kmer_k;
    h.flags = idx->flags;
    memcpy(h.C, idx->C, sizeof h.C);
    u64 cs = checksum_words(&h, offsetof(FileHeader, checksum), 0xCBF29CE484222325ULL);
    for (auto *v : sec) cs = checksum_words(v->data(), v->size(), cs);
    h.checksum = cs;
    FILE *f = fopen(path, "wb");
    if (!f) {
        mb_set_error("mb_index_save: cannot open %s", path);
        return MB_ERR_IO;
    }
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    for (auto *v : sec) ok = ok && fwrite(v->data(), 1, v->size(), f) == v->size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        mb_set_error("mb_index_save: write to %s failed", path);
        return MB_ERR_IO;
    }
    return MB_OK;
}

extern "C" int mb_index_load(const char *path, void *stream, mb_index **out) {
    if (!path || !out) return MB_ERR_ARG;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) {
        mb_set_error("mb_index_load: cannot open %s", path);
        return MB_ERR_IO;
    }
    FileHeader h;
    if (fread(&h, sizeof h, 1, f) != 1) {
        fclose(f);
        mb_set_error("mb_index_load: short header");
        return MB_ERR_CORRUPT;
    }
    if (h.magic != MAGIC || h.version != 4 || h.sa_rate == 0 || h.kmer_k > 16 || h.n >= (1ULL << 32) ||
        h.n < 2 || h.nblocks != h.n / BLK_ROWS + 1) {
        fclose(f);
        mb_set_error("mb_index_load: bad header");
        return MB_ERR_CORRUPT;
    }
    if (h.aux != 0 && h.aux != AUX_RATE) {
        fclose(f);
        mb_set_error("mb_index_load: the file's auxiliary samples are at rate %u, this library reads rate %u "
                     "(rebuild the index)", h.aux, AUX_RATE);
        return MB_ERR_CORRUPT;
    }
    u64 ns = (h.n + h.sa_rate - 1) / h.sa_rate, nk = 1ULL << (2 * h.kmer_k);
    std::vector<u8> occ(h.nblocks * sizeof(OccBlock)), ssa(ns * 4), km(nk * 12);
    std::vector<u8> t2(h.aux ? text2_words(h.n) * 4 : 0), sx(h.aux ? aux_count(h.n) * 4 : 0), ix(sx.size());
    std::vector<u8> *sec[] = {&occ, &ssa, &km, &t2, &sx, &ix};
    bool ok = true;
    for (auto *v : sec) ok = ok && fread(v->data(), 1, v->size(), f) == v->size();
    fclose(f);
    if (!ok) {
        mb_set_error("mb_index_load: truncated file");
        return MB_ERR_CORRUPT;
    }
    u64 cs = checksum_words(&h, offsetof(FileHeader, checksum), 0xCBF29CE484222325ULL);
    for (auto *v : sec) cs = checksum_words(v->data(), v->size(), cs);
    if (cs != h.checksum) {
        mb_set_error("mb_index_load: checksum mismatch");
        return MB_ERR_CORRUPT;
    }
    mb_index *X = new mb_index;
    X->n = h.n;
    X->rlen = h.rlen;
    X->primary = h.primary;
    X->nblocks = h.nblocks;
    X->sa_rate = h.sa_rate;
    X->kmer_k = h.kmer_k;
    X->flags = h.flags;
    memcpy(X->C, h.C, sizeof h.C);
    cudaGetDevice(&X->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMalloc(&X->occ, occ.size()) != cudaSuccess || cudaMalloc(&X->ssa, ssa.size()) != cudaSuccess ||
        cudaMalloc(&X->kmer, km.size()) != cudaSuccess ||
        (h.aux && (cudaMalloc(&X->text2, t2.size()) != cudaSuccess || cudaMalloc(&X->sa_aux, sx.size()) != cudaSuccess ||
                   cudaMalloc(&X->isa_aux, ix.size()) != cudaSuccess))) {
        free_index(X);
        mb_set_error("mb_index_load: device allocation failed");
        return MB_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(X->occ, occ.data(), occ.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(X->ssa, ssa.data(), ssa.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(X->kmer, km.data(), km.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (h.aux && (cudaMemcpyAsync(X->text2, t2.data(), t2.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                   cudaMemcpyAsync(X->sa_aux, sx.data(), sx.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                   cudaMemcpyAsync(X->isa_aux, ix.data(), ix.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)) ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        free_index(X);
        mb_set_error("mb_index_load: copy to device failed");
        return MB_ERR_CUDA;
    }
    *out = X;
    return MB_OK;
}

extern "C" int mb_hit_to_ref(const mb_index *idx, uint64_t pos, uint64_t len, int *strand, uint64_t *rpos) {
    if (!idx || !strand || !rpos || pos + len > idx->n - 1) return MB_ERR_ARG;
    u64 M = idx->rlen;
    if (pos < M) {
        *strand = 0;
        *rpos = pos;
    } else {
        *strand = 1;
        *rpos = 2 * M - pos - len;
    }
    return MB_OK;
}

extern "C" int mb_set_l2_fetch_granularity(int bytes, int *now) {
    if (bytes != 0 && bytes != 32 && bytes != 64 && bytes != 128) return MB_ERR_ARG;
    if (bytes) MB_CK(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes));
    if (now) {
        size_t v = 0;
        MB_CK(cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity));
        *now = (int)v;
    }
    return MB_OK;
}

extern "C" int mb_index_l2_persist(const mb_index *idx, void *stream, uint64_t max_bytes, uint64_t *window) {
    if (!idx || !idx->kmer) return MB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    MB_CK(cudaGetDevice(&dev));
    cudaStreamAttrValue v;
    memset(&v, 0, sizeof v);
    u64 w = 0;
    if (max_bytes) {
        int max_win = 0, max_persist = 0;
        MB_CK(cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev));
        MB_CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
        w = (1ULL << (2 * idx->kmer_k)) * 12;
        if (w > max_bytes) w = max_bytes;
        if (w > (u64)max_win) w = (u64)max_win;
        if (w > (u64)max_persist) w = (u64)max_persist;
        MB_CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)w));
        v.accessPolicyWindow.base_ptr = idx->kmer;
        v.accessPolicyWindow.num_bytes = (size_t)w;
        v.accessPolicyWindow.hitRatio = 1.0f;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    } else {
        v.accessPolicyWindow.num_bytes = 0;   // window off
        MB_CK(cudaCtxResetPersistingL2Cache());
    }
    MB_CK(cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v));
    if (window) *window = w;
    return MB_OK;
}

extern "C" const char *mb_strerror(int code) {
    switch (code) {
    case MB_OK: return "ok";
    case MB_ERR_ARG: return "invalid argument";
    case MB_ERR_NOMEM: return "out of memory";
    case MB_ERR_CAPACITY: return "output buffer too small";
    case MB_ERR_CUDA: return "CUDA error";
    case MB_ERR_TIMEOUT: return "timed out";
    case MB_ERR_IO: return "I/O error";
    case MB_ERR_CORRUPT: return "corrupt index file";
    case MB_ERR_DEVICE_CHECK: return "device-side check failed";
    case MB_ERR_BUSY: return "busy";
    default: return "unknown error";
    }
}
