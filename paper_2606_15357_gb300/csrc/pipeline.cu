// Whole seeding stage with host (or device) buffers in one call: mb_seed_locate.
//
// The batch is cut into chunks of consecutive reads that alternate between two streams.  Each
// stream owns a seeding plan (no host synchronization inside, see mb_plan_run) and device copies
// of its chunk's inputs, so while one stream copies a chunk in, seeds it (Algorithm 3, the
// max-occ flag, Algorithm 2) and copies its records and hits out, the other stream's chunk is on
// the GPU.  Read numbers and hit offsets of a chunk are made global by a small kernel before the
// copy out, so the call returns exactly what mb_seed_batch followed by mb_locate return.
//
// The streams, plans and staging buffers of a call are kept for the next call with the same index,
// device and seeding options whose chunks fit them (at most two sets are kept; they are released
// with the index), so steady-state calls allocate nothing.
#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>
#include "common.cuh"

namespace {

constexpr u32 PIPE_READS = 1u << 22;      // default reads per chunk
constexpr u64 PIPE_BASES = 1ull << 29;    // at most this many bases per chunk (at least one read)
constexpr int PIPE_STAGES = 2;

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
           a.prefetch_depth == b.prefetch_depth && a.block_size == b.block_size;
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

    // offsets on the host to cut the chunks
    std::vector<u64> hoff_copy;
    const u64 *hoff = off;
    if (off_dev) {
        hoff_copy.resize((size_t)n_reads + 1);
        MB_CK(cudaMemcpyAsync(hoff_copy.data(), off, hoff_copy.size() * 8, cudaMemcpyDeviceToHost, ust));
        MB_CK(cudaStreamSynchronize(ust));
        hoff = hoff_copy.data();
    }
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

    // per-stage resources, sized for the largest chunk (a kept set when one fits)
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
        const u64 max_hits = 4ull * max_smem;
        MB_CK(cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming));
        for (Stage &x : p.s) {
            MB_CK(cudaStreamCreateWithFlags(&x.st, cudaStreamNonBlocking));
            MB_CK(cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming));
            MB_CK(cudaMallocHost(&x.hcnt, 16));
            MB_TRY(mb_plan_create(idx, opts, max_nr, max_nb, max_smem, max_hits, &x.plan));
            if (p.own_seq) MB_CK(cudaMalloc(&x.dseq, max_nb + 16));
            if (p.own_off) MB_CK(cudaMalloc(&x.doff, ((size_t)max_nr + 1) * 8));
            if (p.own_mate) MB_CK(cudaMalloc(&x.dmate, max_nr));
        }
    }
    Pipeline &pl = *keep;
    MB_CK(cudaEventRecord(pl.start, ust));
    for (Stage &x : pl.s) MB_CK(cudaStreamWaitEvent(x.st, pl.start, 0));   // after the caller's earlier work

    // inputs of chunk i in, then its whole stage, then its two counts to the host
    auto enqueue = [&](int i, Stage &x) -> int {
        const Chunk &c = chunks[i];
        const u8 *dseq = seq;
        const u64 *doff = off + c.r0;
        const u8 *dmate = mate ? mate + c.r0 : nullptr;
        if (!seq_dev) {
            if (c.o1 > c.o0) MB_CK(cudaMemcpyAsync(x.dseq, seq + c.o0, c.o1 - c.o0, cudaMemcpyHostToDevice, x.st));
            dseq = x.dseq - c.o0;   // read r of the chunk starts at dseq + off[r], as in the caller's buffer
        }
        if (!off_dev) {
            MB_CK(cudaMemcpyAsync(x.doff, off + c.r0, ((size_t)c.nr + 1) * 8, cudaMemcpyHostToDevice, x.st));
            doff = x.doff;
        }
        if (mate && !mate_dev) {
            MB_CK(cudaMemcpyAsync(x.dmate, mate + c.r0, c.nr, cudaMemcpyHostToDevice, x.st));
            dmate = x.dmate;
        }
        MB_TRY(mb_plan_run(x.plan, dseq, doff, c.nr, dmate, x.st));
        MB_TRY(mb_plan_counts_async(x.plan, x.hcnt, x.st));
        MB_CK(cudaEventRecord(x.ev, x.st));
        x.chunk = i;
        return MB_OK;
    };

    u64 m_tot = 0, h_tot = 0;
    bool over = false;
    // chunk i's counts are on the host: its records and hits out (no wait on the copies)
    auto drain = [&](Stage &x) -> int {
        const Chunk &c = chunks[x.chunk];
        MB_CK(cudaEventSynchronize(x.ev));
        u64 ns = x.hcnt[0], nh = x.hcnt[1];
        const mb_smem *psm;
        const u32 *ph;
        u64 ms, mh;
        mb_plan_arrays(x.plan, &psm, &ph, &ms, &mh);
        DevBuf fsm, fh;
        if (ns > ms || nh > mh) {
            // the chunk outgrew the plan: the allocating path on the chunk's device inputs
            const u8 *dseq = seq_dev ? seq : x.dseq - c.o0;
            const u64 *doff = off_dev ? off + c.r0 : x.doff;
            const u8 *dmate = mate ? (mate_dev ? mate + c.r0 : x.dmate) : nullptr;
            u64 h = 0;
            MB_TRY(fsm.alloc(ns * sizeof(mb_smem) + 64, x.st));
            MB_TRY(mb_seed_batch(idx, dseq, doff, c.nr, dmate, opts, x.st, fsm.as<mb_smem>(), ns, &ns, &h));
            MB_TRY(fh.alloc(h * 4 + 64, x.st));
            MB_TRY(mb_locate(idx, fsm.as<mb_smem>(), ns, opts, x.st, fh.as<u32>(), h, &nh));
            psm = fsm.as<mb_smem>();
            ph = fh.as<u32>();
        }
        if (!over && (m_tot + ns > cap || h_tot + nh > hits_cap || (ns && !out) || (nh && !hits))) over = true;
        if (!over) {
            if (ns) {
                k_rebase<<<grid_for(ns, 256), 256, 0, x.st>>>((mb_smem *)psm, ns, c.r0, h_tot);
                MB_KCHECK();
                MB_CK(cudaMemcpyAsync(out + m_tot, psm, ns * sizeof(mb_smem), cudaMemcpyDefault, x.st));
            }
            if (nh) MB_CK(cudaMemcpyAsync(hits + h_tot, ph, nh * 4, cudaMemcpyDefault, x.st));
        }
        m_tot += ns;
        h_tot += nh;
        x.chunk = -1;
        return MB_OK;   // a fallback's buffers are freed in stream order after the copies
    };

    const int nc = (int)chunks.size();
    for (int i = 0; i < nc && i < PIPE_STAGES; ++i) MB_TRY(enqueue(i, pl.s[i]));
    for (int i = 0; i < nc; ++i) {
        Stage &x = pl.s[i % PIPE_STAGES];
        MB_TRY(drain(x));
        if (i + PIPE_STAGES < nc) MB_TRY(enqueue(i + PIPE_STAGES, x));
    }
    for (Stage &x : pl.s) MB_CK(cudaStreamSynchronize(x.st));
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
