// Whole seeding stage with host (or device) buffers in one call: mb_seed_locate.
//
// The batch is cut into slices of at most 2^25 reads and 2^33 bases, and a slice into chunks of
// consecutive reads that alternate between two streams.  Each stream owns a seeding plan (no host
// synchronization inside) and device copies of its chunk's inputs, so while one stream copies a
// chunk in and seeds it (Algorithm 3 and the max-occ flag, up to the records and their hit
// offsets), the other stream's chunk is on the GPU.  A chunk's records, with read numbers and hit
// offsets made slice-wide by a small kernel, and the positions found while seeding are gathered
// in device arrays of the slice; then the slice is located at once (Algorithm 2, every distinct
// row walked once, so the repeats of the whole slice share their walks) while its records are
// copied out on the other stream, and its hits are copied out last.  The call returns exactly
// what mb_seed_batch followed by mb_locate return.
//
// The streams, plans and staging buffers of a call are kept for the next call with the same index,
// device and seeding options whose chunks fit them (at most two sets are kept; they are released
// with the index).
#include <algorithm>
#include <cstdlib>
#include <memory>
#include <mutex>
#include <vector>
#include "common.cuh"

namespace {

constexpr u32 PIPE_READS = 1u << 22;      // default reads per chunk
constexpr u64 PIPE_BASES = 1ull << 29;    // at most this many bases per chunk (at least one read)
constexpr u32 SLICE_READS = 1u << 25;     // at most this many reads per slice (located at once)
                                          // (MB_SLICE_READS in the environment may lower it)
constexpr u64 SLICE_BASES = 1ull << 33;   // and this many bases (at least one chunk)
constexpr int PIPE_STAGES = 2;

u32 slice_reads() {
    const char *e = getenv("MB_SLICE_READS");
    if (e) {
        const long v = atol(e);
        if (v > 0 && v < (long)SLICE_READS) return (u32)v;
    }
    return SLICE_READS;
}

// records of one chunk in batch coordinates: read number and first hit
__global__ void k_rebase(mb_smem *__restrict__ s, u64 n, u32 r0, u64 h0) {
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < n; t += (u64)gridDim.x * blockDim.x) {
        s[t].read += r0;
        s[t].hit_off += h0;
    }
}

struct Chunk {
    u32 r0 = 0, nr = 0;
    u64 o0 = 0, o1 = 0;
};
struct Slice {
    int c0 = 0, c1 = 0;   // its chunks [c0, c1)
    u64 cap = 0;          // records its chunks' plans hold
};

struct Stage {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    mb_plan *plan = nullptr;
    u8 *dseq = nullptr, *dmate = nullptr;   // chunk copies (host inputs only)
    u64 *doff = nullptr;
    u64 *hcnt = nullptr;                    // pinned: n_smem, n_hits of the chunk in flight
    int chunk = -1;
};

struct Pipeline {
    const mb_index *idx = nullptr;
    int device = -1;
    mb_opts opts{};                // options the plans were made with
    u32 max_nr = 0;                // capacity: reads and bases per chunk
    u64 max_nb = 0;
    bool own_seq = false, own_off = false, own_mate = false;   // staging buffers present
    Stage s[PIPE_STAGES];
    cudaEvent_t start = nullptr;   // recorded on the caller's stream
    ~Pipeline() {
        if (start) cudaEventDestroy(start);
        for (Stage &x : s) {
            if (x.st) cudaStreamSynchronize(x.st);
            if (x.plan) mb_plan_free(x.plan);
            if (x.dseq) cudaFree(x.dseq);
            if (x.dmate) cudaFree(x.dmate);
            if (x.doff) cudaFree(x.doff);
            if (x.hcnt) cudaFreeHost(x.hcnt);
            if (x.ev) cudaEventDestroy(x.ev);
            if (x.st) cudaStreamDestroy(x.st);
        }
    }
};

// the options that shape a plan (chunk_reads only sizes the chunks)
bool same_plan_opts(const mb_opts &a, const mb_opts &b) {
    return a.min_len == b.min_len && a.min_occ == b.min_occ && a.max_occ == b.max_occ && a.flags == b.flags &&
           a.prefetch_depth == b.prefetch_depth && a.block_size == b.block_size && a.smem_burst == b.smem_burst &&
           a.smem_wait == b.smem_wait && a.smem_warps == b.smem_warps &&
           a.smem_reads_per_warp == b.smem_reads_per_warp;
}

constexpr size_t KEEP = 2;
std::mutex g_mu;
std::vector<std::unique_ptr<Pipeline>> g_idle;

std::unique_ptr<Pipeline> take_pipeline(const mb_index *idx, int device, const mb_opts &o, u32 nr, u64 nb,
                                        bool seq, bool off, bool mate) {
    std::lock_guard<std::mutex> g(g_mu);
    for (size_t i = 0; i < g_idle.size(); ++i) {
        Pipeline &p = *g_idle[i];
        if (p.idx == idx && p.device == device && same_plan_opts(p.opts, o) && p.max_nr >= nr && p.max_nb >= nb &&
            (p.own_seq || !seq) && (p.own_off || !off) && (p.own_mate || !mate)) {
            std::unique_ptr<Pipeline> r = std::move(g_idle[i]);
            g_idle.erase(g_idle.begin() + i);
            return r;
        }
    }
    return nullptr;
}

void keep_pipeline(std::unique_ptr<Pipeline> p) {
    std::unique_ptr<Pipeline> drop;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_idle.push_back(std::move(p));
        if (g_idle.size() > KEEP) {
            drop = std::move(g_idle.front());
            g_idle.erase(g_idle.begin());
        }
    }
}

}  // namespace

void mb_pipeline_forget(const mb_index *idx) {
    std::vector<std::unique_ptr<Pipeline>> drop;
    std::lock_guard<std::mutex> g(g_mu);
    for (size_t i = 0; i < g_idle.size();) {
        if (g_idle[i]->idx == idx) {
            drop.push_back(std::move(g_idle[i]));
            g_idle.erase(g_idle.begin() + i);
        } else {
            ++i;
        }
    }
}

extern "C" int mb_seed_locate(const mb_index *idx, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                              const uint8_t *mate, const mb_opts *opts, void *stream, mb_smem *out, uint64_t cap,
                              uint32_t *hits, uint64_t hits_cap, uint64_t *n_out, uint64_t *n_hits) {
    if (!idx || !off || !n_out || !n_hits || (n_reads > 0 && !seq)) {
        mb_set_error("mb_seed_locate: null argument");
        return MB_ERR_ARG;
    }
    *n_out = 0;
    *n_hits = 0;
    if (n_reads == 0) return MB_OK;
    cudaStream_t ust = (cudaStream_t)stream;
    const bool seq_dev = mb_is_device_ptr(seq), off_dev = mb_is_device_ptr(off);
    const bool mate_dev = mate && mb_is_device_ptr(mate);

    // device buffers must hold what the call reads and writes (checked before any access)
    MB_TRY(mb_check_span(off, ((size_t)n_reads + 1) * 8, "mb_seed_locate: off"));
    if (mate) MB_TRY(mb_check_span(mate, n_reads, "mb_seed_locate: mate"));
    if (out) MB_TRY(mb_check_span(out, cap * sizeof(mb_smem), "mb_seed_locate: out"));
    if (hits) MB_TRY(mb_check_span(hits, hits_cap * 4, "mb_seed_locate: hits"));
    // offsets on the host to cut the chunks
    std::vector<u64> hoff_copy;
    const u64 *hoff = off;
    if (off_dev) {
        hoff_copy.resize((size_t)n_reads + 1);
        MB_CK(cudaMemcpyAsync(hoff_copy.data(), off, hoff_copy.size() * 8, cudaMemcpyDeviceToHost, ust));
        MB_CK(cudaStreamSynchronize(ust));
        hoff = hoff_copy.data();
    }
    if (hoff[n_reads] < hoff[0]) {
        mb_set_error("mb_seed_locate: offsets decrease");
        return MB_ERR_ARG;
    }
    MB_TRY(mb_check_span(seq + hoff[0], hoff[n_reads] - hoff[0], "mb_seed_locate: seq[off[0], off[n_reads])"));
    const u32 per = opts && opts->chunk_reads ? opts->chunk_reads : PIPE_READS;
    std::vector<Chunk> chunks;
    u32 max_nr = 0;
    u64 max_nb = 0;
    for (u32 r = 0; r < n_reads;) {
        Chunk c;
        c.r0 = r;
        c.o0 = hoff[r];
        // the chunk ends before the first read (after read r) whose end passes o0 + PIPE_BASES, and
        // after at most `per` reads: a binary search over the offsets (which must not decrease)
        const u32 emax = (u32)std::min<u64>((u64)n_reads, (u64)r + per);
        const u64 lim = c.o0 + PIPE_BASES;
        u32 e = (u32)(std::upper_bound(hoff + r + 2, hoff + emax + 1, lim) - (hoff + 1));
        if (e < r + 1) e = r + 1;
        c.nr = e - r;
        c.o1 = hoff[e];
        if (c.o1 < c.o0) {
            mb_set_error("mb_seed_locate: offsets decrease at read %u", r);
            return MB_ERR_ARG;
        }
        if (c.nr > max_nr) max_nr = c.nr;
        if (c.o1 - c.o0 > max_nb) max_nb = c.o1 - c.o0;
        chunks.push_back(c);
        r = e;
    }

    // slices: consecutive chunks up to slice_reads() reads and SLICE_BASES bases
    const u32 max_slice = slice_reads();
    std::vector<Slice> slices;
    for (int i = 0; i < (int)chunks.size();) {
        Slice sl;
        sl.c0 = i;
        u64 nr = 0, nb = 0;
        while (i < (int)chunks.size() && (i == sl.c0 || (nr + chunks[i].nr <= max_slice &&
                                                         nb + (chunks[i].o1 - chunks[i].o0) <= SLICE_BASES))) {
            nr += chunks[i].nr;
            nb += chunks[i].o1 - chunks[i].o0;
            sl.cap += 4ull * chunks[i].nr + (chunks[i].o1 - chunks[i].o0) / 32 + 64;
            ++i;
        }
        sl.c1 = i;
        slices.push_back(sl);
    }

    // per-stage resources, sized for the largest chunk (a kept set when one fits); the plans only
    // seed, so they hold no hits
    int device = 0;
    MB_CK(cudaGetDevice(&device));
    const mb_opts o = opts ? *opts : mb_opts{};
    std::unique_ptr<Pipeline> keep =
        take_pipeline(idx, device, o, max_nr, max_nb, !seq_dev, !off_dev, mate && !mate_dev);
    if (!keep) {
        keep.reset(new Pipeline);
        Pipeline &p = *keep;
        p.idx = idx;
        p.device = device;
        p.opts = o;
        p.max_nr = max_nr;
        p.max_nb = max_nb;
        p.own_seq = !seq_dev;
        p.own_off = !off_dev;
        p.own_mate = mate && !mate_dev;
        const u64 max_smem = 4ull * max_nr + max_nb / 32 + 64;
        MB_CK(cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming));
        for (Stage &x : p.s) {
            MB_CK(cudaStreamCreateWithFlags(&x.st, cudaStreamNonBlocking));
            MB_CK(cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming));
            MB_CK(cudaMallocHost(&x.hcnt, 32));
            MB_TRY(mb_plan_create(idx, opts, max_nr, max_nb, max_smem, 1, &x.plan));
            if (p.own_seq) MB_CK(cudaMalloc(&x.dseq, max_nb + 16));
            if (p.own_off) MB_CK(cudaMalloc(&x.doff, ((size_t)max_nr + 1) * 8));
            if (p.own_mate) MB_CK(cudaMalloc(&x.dmate, max_nr));
        }
    }
    Pipeline &pl = *keep;
    Stage &A = pl.s[0], &B = pl.s[1];
    const bool hits_dev = hits && mb_is_device_ptr(hits);
    const u32 depth = opts ? opts->prefetch_depth : 0;
    const bool join = opts && (opts->flags & MB_LOCATE_JOIN) && !(opts->flags & MB_CHECKED);
    const bool aux = opts && (opts->flags & MB_LOCATE_AUX);

    // device inputs of chunk i (the caller's, or the stage's copies)
    auto inputs = [&](int i, const Stage &x, const u8 *&dseq, const u64 *&doff, const u8 *&dmate) {
        const Chunk &c = chunks[i];
        dseq = seq_dev ? seq : x.dseq - c.o0;   // read r of the chunk starts at dseq + off[r]
        doff = off_dev ? off + c.r0 : x.doff;
        dmate = mate ? (mate_dev ? mate + c.r0 : x.dmate) : nullptr;
    };

    u64 m_tot = 0, h_tot = 0;   // over the whole batch
    bool over = false;
    for (const Slice &sl : slices) {
        // the slice's records and known positions, gathered on the device
        DevBuf gsm, gknown;
        u64 gcap = sl.cap;
        MB_TRY(gsm.alloc(gcap * sizeof(mb_smem), ust));
        MB_TRY(gknown.alloc(gcap * 4, ust));
        MB_CK(cudaEventRecord(pl.start, ust));
        for (Stage &x : pl.s) MB_CK(cudaStreamWaitEvent(x.st, pl.start, 0));   // after the caller's work and the allocations

        // inputs of chunk i in, then its seeding, then its two counts to the host
        auto enqueue = [&](int i, Stage &x) -> int {
            const Chunk &c = chunks[i];
            if (!seq_dev && c.o1 > c.o0)
                MB_CK(cudaMemcpyAsync(x.dseq, seq + c.o0, c.o1 - c.o0, cudaMemcpyHostToDevice, x.st));
            if (!off_dev)
                MB_CK(cudaMemcpyAsync(x.doff, off + c.r0, ((size_t)c.nr + 1) * 8, cudaMemcpyHostToDevice, x.st));
            if (mate && !mate_dev) MB_CK(cudaMemcpyAsync(x.dmate, mate + c.r0, c.nr, cudaMemcpyHostToDevice, x.st));
            const u8 *dseq, *dmate;
            const u64 *doff;
            inputs(i, x, dseq, doff, dmate);
            MB_TRY(mb_plan_run_seed(x.plan, dseq, doff, c.nr, dmate, x.st));
            MB_TRY(mb_plan_counts_async(x.plan, x.hcnt, x.st));
            MB_CK(cudaEventRecord(x.ev, x.st));
            x.chunk = i;
            return MB_OK;
        };

        u64 ms_tot = 0, hs_tot = 0;   // within the slice
        // chunk i's counts are on the host: its records, slice-wide, and known positions gathered
        auto drain = [&](Stage &x) -> int {
            const Chunk &c = chunks[x.chunk];
            MB_CK(cudaEventSynchronize(x.ev));
            if (x.hcnt[2] >> 32) {
                mb_set_error("mb_seed_locate: device check failed (0x%x): read offsets decrease or leave the chunk",
                             (unsigned)(x.hcnt[2] >> 32));
                return MB_ERR_DEVICE_CHECK;
            }
            u64 ns = x.hcnt[0], nh = x.hcnt[1];
            const mb_smem *psm;
            const u32 *ph;
            u64 ms, mh;
            mb_plan_arrays(x.plan, &psm, &ph, &ms, &mh);
            const u32 *pknown = mb_plan_known(x.plan);
            DevBuf fsm;
            if (ns > ms) {
                // the chunk outgrew the plan: the allocating path on the chunk's device inputs (no
                // positions known from seeding)
                const u8 *dseq, *dmate;
                const u64 *doff;
                inputs(x.chunk, x, dseq, doff, dmate);
                MB_TRY(fsm.alloc(ns * sizeof(mb_smem) + 64, x.st));
                // the chunk's inputs are device arrays (dseq may point before the stage's copy,
                // so nothing here is classified by address)
                MB_TRY(mb_seed_device(idx, dseq, doff, c.nr, dmate, nullptr, c.o0, c.o1, opts, x.st,
                                      fsm.as<mb_smem>(), ns, &ns, &nh));
                psm = fsm.as<mb_smem>();
                pknown = nullptr;
            }
            if (ms_tot + ns > gcap) {   // only after the allocating path: grow the slice's arrays
                for (Stage &y : pl.s) MB_CK(cudaStreamSynchronize(y.st));
                const u64 ncap = 2 * (ms_tot + ns);
                DevBuf nsm, nkn;
                MB_TRY(nsm.alloc(ncap * sizeof(mb_smem), x.st));
                MB_TRY(nkn.alloc(ncap * 4, x.st));
                if (ms_tot) {
                    MB_CK(cudaMemcpyAsync(nsm.p, gsm.p, ms_tot * sizeof(mb_smem), cudaMemcpyDeviceToDevice, x.st));
                    MB_CK(cudaMemcpyAsync(nkn.p, gknown.p, ms_tot * 4, cudaMemcpyDeviceToDevice, x.st));
                }
                MB_CK(cudaStreamSynchronize(x.st));
                std::swap(gsm.p, nsm.p);
                std::swap(gsm.bytes, nsm.bytes);
                std::swap(gsm.st, nsm.st);
                std::swap(gknown.p, nkn.p);
                std::swap(gknown.bytes, nkn.bytes);
                std::swap(gknown.st, nkn.st);
                gcap = ncap;
            }
            if (ns) {
                k_rebase<<<grid_for(ns, 256), 256, 0, x.st>>>((mb_smem *)psm, ns, c.r0, hs_tot);
                MB_KCHECK();
                MB_CK(cudaMemcpyAsync(gsm.as<mb_smem>() + ms_tot, psm, ns * sizeof(mb_smem), cudaMemcpyDeviceToDevice,
                                      x.st));
                if (pknown) MB_CK(cudaMemcpyAsync(gknown.as<u32>() + ms_tot, pknown, ns * 4, cudaMemcpyDeviceToDevice, x.st));
                else MB_CK(cudaMemsetAsync(gknown.as<u32>() + ms_tot, 0xFF, ns * 4, x.st));
            }
            ms_tot += ns;
            hs_tot += nh;
            x.chunk = -1;
            return MB_OK;   // a fallback's buffer is freed in stream order after the copy
        };

        const int nc = sl.c1 - sl.c0;
        for (int i = 0; i < nc && i < PIPE_STAGES; ++i) MB_TRY(enqueue(sl.c0 + i, pl.s[i]));
        for (int i = 0; i < nc; ++i) {
            Stage &x = pl.s[i % PIPE_STAGES];
            MB_TRY(drain(x));
            if (i + PIPE_STAGES < nc) MB_TRY(enqueue(sl.c0 + i + PIPE_STAGES, x));
        }
        for (Stage &x : pl.s) MB_CK(cudaStreamSynchronize(x.st));

        // locate the slice at once (stream A) while its records go out (stream B), hits last
        if (!over && (m_tot + ms_tot > cap || h_tot + hs_tot > hits_cap || (ms_tot && !out) || (hs_tot && !hits)))
            over = true;
        if (!over && ms_tot) {
            DevBuf dh;
            u32 *dhits = hits_dev ? hits + h_tot : nullptr;
            if (!hits_dev && hs_tot) {
                MB_TRY(dh.alloc(hs_tot * 4, A.st));
                dhits = dh.as<u32>();
            }
            if (h_tot == 0)   // hit offsets are already batch-wide: copy the records out now
                MB_CK(cudaMemcpyAsync(out + m_tot, gsm.p, ms_tot * sizeof(mb_smem), cudaMemcpyDefault, B.st));
            MB_TRY(mb_locate_records(idx, gsm.as<mb_smem>(), ms_tot, gknown.as<u32>(), dhits, hs_tot, depth, join,
                                     aux, A.st));
            if (h_tot) {      // later slices: batch-wide hit offsets after the locate
                k_rebase<<<grid_for(ms_tot, 256), 256, 0, A.st>>>(gsm.as<mb_smem>(), ms_tot, 0, h_tot);
                MB_KCHECK();
                MB_CK(cudaMemcpyAsync(out + m_tot, gsm.p, ms_tot * sizeof(mb_smem), cudaMemcpyDefault, A.st));
            }
            if (!hits_dev && hs_tot) MB_CK(cudaMemcpyAsync(hits + h_tot, dhits, hs_tot * 4, cudaMemcpyDeviceToHost, A.st));
            MB_CK(cudaStreamSynchronize(A.st));
            MB_CK(cudaStreamSynchronize(B.st));
        }
        m_tot += ms_tot;
        h_tot += hs_tot;
        // the slice's arrays are freed on the caller's stream, after the stage streams' work above
        MB_CK(cudaEventRecord(A.ev, A.st));
        MB_CK(cudaStreamWaitEvent(ust, A.ev, 0));
        MB_CK(cudaEventRecord(B.ev, B.st));
        MB_CK(cudaStreamWaitEvent(ust, B.ev, 0));
    }
    keep_pipeline(std::move(keep));
    *n_out = m_tot;
    *n_hits = h_tot;
    if (over) {
        if (m_tot > cap || h_tot > hits_cap) return MB_ERR_CAPACITY;
        mb_set_error("mb_seed_locate: null output");
        return MB_ERR_ARG;
    }
    return MB_OK;
}
