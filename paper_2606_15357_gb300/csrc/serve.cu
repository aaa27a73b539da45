// Served form: continuous batching of seeding requests (the whole stage of Section 2.5 and
// Algorithm 2 per request) on one GPU.
//
// A worker thread owns a set of execution slots (a stream, a seeding plan and pinned staging
// buffers each, as many as fit the HBM budget).  Whenever a slot is free it merges every waiting
// request that still fits the slot's limits into one launch group, copies the group in, runs the
// plan and records an event; completion is handled in two asynchronous phases (the two result
// counts, then the results themselves), so the worker never blocks on the GPU and groups on
// different slots overlap on the device.  Each request gets back exactly what mb_seed_batch +
// mb_locate give for it alone: read numbers and hit offsets are made relative to the request.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include "common.cuh"

namespace {

constexpr u32 SLOT_READS = 65536;
constexpr u64 SLOT_BASES = 64ull << 20;
constexpr u64 SLOT_SMEM = 2ull << 20;
constexpr u64 SLOT_HITS = 32ull << 20;
constexpr int MAX_SLOTS = 16;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    u64 ticket = 0;
    std::vector<u8> seq;
    std::vector<u64> off;   // n_reads + 1, from 0
    u32 n_reads = 0;
    double t_submit = 0, latency_ms = 0;
    bool done = false;
    int status = MB_OK;
    std::vector<mb_smem> smem;
    std::vector<u32> hits;
};
using ReqP = std::shared_ptr<Request>;

enum Phase { IDLE, RUNNING, COPYING };

struct Slot {
    cudaStream_t st = nullptr;
    mb_plan *plan = nullptr;
    u8 *dseq = nullptr;
    u64 *doff = nullptr;
    u8 *hseq = nullptr;       // pinned
    u64 *hoff = nullptr;      // pinned
    u64 *hcnt = nullptr;      // pinned: n_smem, n_hits
    mb_smem *hsmem = nullptr; // pinned
    u32 *hhits = nullptr;     // pinned
    cudaEvent_t ev = nullptr;
    Phase phase = IDLE;
    std::vector<ReqP> group;
    std::vector<u32> first_read;   // first group read of each request
    u32 n_reads = 0;
};

}  // namespace

struct mb_server {
    const mb_index *idx = nullptr;
    mb_opts opts{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ReqP> pending;
    std::unordered_map<u64, ReqP> reqs;
    std::thread worker;
    bool stop = false;
    u64 next_ticket = 1;
    u64 groups = 0, merged = 0;
    int device = 0;
};

namespace {

void free_slot(Slot &s) {
    if (s.plan) mb_plan_free(s.plan);
    if (s.dseq) cudaFree(s.dseq);
    if (s.doff) cudaFree(s.doff);
    if (s.hseq) cudaFreeHost(s.hseq);
    if (s.hoff) cudaFreeHost(s.hoff);
    if (s.hcnt) cudaFreeHost(s.hcnt);
    if (s.hsmem) cudaFreeHost(s.hsmem);
    if (s.hhits) cudaFreeHost(s.hhits);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.st) cudaStreamDestroy(s.st);
    s = Slot{};
}

int make_slot(mb_server *S, Slot &s) {
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess)
        return MB_ERR_CUDA;
    MB_TRY(mb_plan_create(S->idx, &S->opts, SLOT_READS, SLOT_BASES, SLOT_SMEM, SLOT_HITS, &s.plan));
    if (cudaMalloc(&s.dseq, SLOT_BASES) != cudaSuccess || cudaMalloc(&s.doff, (SLOT_READS + 1) * 8) != cudaSuccess ||
        cudaMallocHost(&s.hseq, SLOT_BASES) != cudaSuccess || cudaMallocHost(&s.hoff, (SLOT_READS + 1) * 8) != cudaSuccess ||
        cudaMallocHost(&s.hcnt, 16) != cudaSuccess || cudaMallocHost(&s.hsmem, SLOT_SMEM * sizeof(mb_smem)) != cudaSuccess ||
        cudaMallocHost(&s.hhits, SLOT_HITS * 4) != cudaSuccess) {
        cudaGetLastError();
        return MB_ERR_NOMEM;
    }
    return MB_OK;
}

size_t slot_device_bytes(const Slot &s) { return mb_plan_bytes(s.plan) + SLOT_BASES + (SLOT_READS + 1) * 8; }

// Merge waiting requests into the free slot s (called with the lock held).  Returns false if
// nothing is waiting.
bool admit(mb_server *S, Slot &s) {
    if (S->pending.empty()) return false;
    s.group.clear();
    s.first_read.clear();
    u32 nr = 0;
    u64 nb = 0;
    while (!S->pending.empty()) {
        const ReqP &r = S->pending.front();
        const u64 b = r->off[r->n_reads];
        if (!s.group.empty() && (nr + r->n_reads > SLOT_READS || nb + b > SLOT_BASES)) break;
        s.first_read.push_back(nr);
        s.group.push_back(r);
        nr += r->n_reads;
        nb += b;
        S->pending.pop_front();
    }
    s.n_reads = nr;
    return true;
}

// Copy the group in and run it (lock not held).
int launch(mb_server *S, Slot &s) {
    u64 nb = 0;
    u32 nr = 0;
    s.hoff[0] = 0;
    for (const ReqP &r : s.group) {
        memcpy(s.hseq + nb, r->seq.data(), r->seq.size());
        for (u32 i = 0; i < r->n_reads; ++i) s.hoff[nr + i + 1] = nb + r->off[i + 1];
        nb += r->seq.size();
        nr += r->n_reads;
    }
    MB_CK(cudaMemcpyAsync(s.dseq, s.hseq, nb ? nb : 1, cudaMemcpyHostToDevice, s.st));
    MB_CK(cudaMemcpyAsync(s.doff, s.hoff, (size_t)(nr + 1) * 8, cudaMemcpyHostToDevice, s.st));
    MB_TRY(mb_plan_run(s.plan, s.dseq, s.doff, nr, nullptr, s.st));
    MB_TRY(mb_plan_counts_async(s.plan, s.hcnt, s.st));
    MB_CK(cudaEventRecord(s.ev, s.st));
    s.phase = RUNNING;
    return MB_OK;
}

// The group's counts are on the host: copy the results back (or fall back when a limit was hit).
int fetch(mb_server *S, Slot &s) {
    const u64 ns = s.hcnt[0], nh = s.hcnt[1];
    const mb_smem *dsm;
    const u32 *dh;
    u64 ms, mh;
    mb_plan_arrays(s.plan, &dsm, &dh, &ms, &mh);
    if (ns > ms || nh > mh) {
        // the merged group outgrew the plan: seed its requests one by one with the allocating path
        for (const ReqP &r : s.group) {
            u64 m = 0, h = 0;
            int rc = mb_seed_batch(S->idx, r->seq.data(), r->off.data(), r->n_reads, nullptr, &S->opts, s.st, nullptr,
                                   0, &m, &h);
            if (rc != MB_OK && rc != MB_ERR_CAPACITY) { r->status = rc; continue; }
            r->smem.resize(m);
            rc = mb_seed_batch(S->idx, r->seq.data(), r->off.data(), r->n_reads, nullptr, &S->opts, s.st,
                               r->smem.data(), m, &m, &h);
            if (rc == MB_OK) {
                r->hits.resize(h);
                rc = mb_locate(S->idx, r->smem.data(), m, &S->opts, s.st, r->hits.data(), h, &h);
            }
            r->status = rc;
        }
        s.phase = IDLE;
        return 1;   // results are final
    }
    if (ns) MB_CK(cudaMemcpyAsync(s.hsmem, dsm, ns * sizeof(mb_smem), cudaMemcpyDeviceToHost, s.st));
    if (nh) MB_CK(cudaMemcpyAsync(s.hhits, dh, nh * 4, cudaMemcpyDeviceToHost, s.st));
    MB_CK(cudaEventRecord(s.ev, s.st));
    s.phase = COPYING;
    return 0;
}

// Split the group's records and hits per request, relative to each request.
void split(Slot &s) {
    const u64 ns = s.hcnt[0], nh = s.hcnt[1];
    u64 m = 0;
    for (size_t q = 0; q < s.group.size(); ++q) {
        Request &r = *s.group[q];
        const u32 r0 = s.first_read[q], r1 = r0 + r.n_reads;
        const u64 m0 = m;
        while (m < ns && s.hsmem[m].read < r1) ++m;
        const u64 h0 = m0 < ns ? s.hsmem[m0].hit_off : nh;
        const u64 h1 = m < ns ? s.hsmem[m].hit_off : nh;
        r.smem.assign(s.hsmem + m0, s.hsmem + m);
        for (mb_smem &x : r.smem) {
            x.read -= r0;
            x.hit_off -= h0;
        }
        r.hits.assign(s.hhits + h0, s.hhits + h1);
        r.status = MB_OK;
    }
}

void finish(mb_server *S, Slot &s) {
    const double t = now_ms();
    std::lock_guard<std::mutex> g(S->mu);
    for (const ReqP &r : s.group) {
        r->latency_ms = t - r->t_submit;
        r->done = true;
    }
    S->groups += 1;
    if (s.group.size() > 1) S->merged += s.group.size();
    s.group.clear();
    s.phase = IDLE;
    S->cv.notify_all();
}

void worker_loop(mb_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool any_busy = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (Slot &s : S->slots) any_busy |= s.phase != IDLE;
            if (S->stop && S->pending.empty() && !any_busy) return;
            if (S->pending.empty() && !any_busy) {
                S->cv.wait(lk, [&] { return S->stop || !S->pending.empty(); });
                continue;
            }
        }
        bool progressed = false;
        for (Slot &s : S->slots) {
            if (s.phase == IDLE) {
                bool got;
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    got = admit(S, s);
                }
                if (got) {
                    if (launch(S, s) != MB_OK) {
                        for (const ReqP &r : s.group) r->status = MB_ERR_CUDA;
                        finish(S, s);
                    }
                    progressed = true;
                }
            } else if (cudaEventQuery(s.ev) == cudaSuccess) {
                if (s.phase == RUNNING) {
                    int rc = fetch(S, s);
                    if (rc == 1) finish(S, s);
                    else if (rc != MB_OK) {
                        for (const ReqP &r : s.group) r->status = rc;
                        finish(S, s);
                    }
                } else {
                    split(s);
                    finish(S, s);
                }
                progressed = true;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" int mb_serve_create(const mb_index *idx, const mb_opts *opts, uint64_t hbm_budget, mb_server **out) {
    if (!idx || !out) return MB_ERR_ARG;
    *out = nullptr;
    mb_server *S = new mb_server;
    S->idx = idx;
    if (opts) S->opts = *opts;
    S->opts.flags |= MB_BATCHED;
    S->opts.flags &= ~(u32)MB_COUNT;
    cudaGetDevice(&S->device);
    u64 used = 0;
    for (int i = 0; i < MAX_SLOTS; ++i) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        Slot s;
        int rc = make_slot(S, s);
        if (rc != MB_OK) {
            free_slot(s);
            if (i == 0) {
                delete S;
                mb_set_error("mb_serve_create: cannot create one execution slot");
                return rc;
            }
            break;
        }
        const u64 b = slot_device_bytes(s);
        if (i > 0 && used + b > hbm_budget) {
            free_slot(s);
            break;
        }
        used += b;
        S->slots.push_back(s);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return MB_OK;
}

extern "C" int mb_serve_submit(mb_server *S, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                               uint64_t *ticket) {
    if (!S || !ticket || !off || (n_reads && !seq)) return MB_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->n_reads = n_reads;
    r->off.resize((size_t)n_reads + 1);
    for (u32 i = 0; i <= n_reads; ++i) r->off[i] = off[i] - off[0];
    const u64 nb = r->off[n_reads];
    if (n_reads > SLOT_READS || nb > SLOT_BASES) {
        mb_set_error("mb_serve_submit: %u reads / %llu bases exceed one slot (%u / %llu)", n_reads,
                     (unsigned long long)nb, SLOT_READS, (unsigned long long)SLOT_BASES);
        return MB_ERR_ARG;
    }
    r->seq.assign(seq + off[0], seq + off[0] + nb);
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return MB_ERR_ARG;
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    *ticket = r->ticket;
    S->cv.notify_all();
    return MB_OK;
}

extern "C" int mb_serve_poll(mb_server *S, uint64_t ticket, int *done) {
    if (!S || !done) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MB_ERR_ARG;
    *done = it->second->done ? 1 : 0;
    return MB_OK;
}

extern "C" int mb_serve_wait(mb_server *S, uint64_t ticket, uint32_t timeout_ms, const mb_smem **smem,
                             uint64_t *n_smem, const uint32_t **hits, uint64_t *n_hits, double *latency_ms) {
    if (!S) return MB_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MB_ERR_ARG;
    ReqP r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms == 0) S->cv.wait(lk, ready);
    else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return MB_ERR_TIMEOUT;
    if (r->status != MB_OK) return r->status;
    if (smem) *smem = r->smem.data();
    if (n_smem) *n_smem = r->smem.size();
    if (hits) *hits = r->hits.data();
    if (n_hits) *n_hits = r->hits.size();
    if (latency_ms) *latency_ms = r->latency_ms;
    return MB_OK;
}

extern "C" int mb_serve_release(mb_server *S, uint64_t ticket) {
    if (!S) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->done) return MB_ERR_ARG;
    S->reqs.erase(it);
    return MB_OK;
}

extern "C" int mb_serve_stats(mb_server *S, uint32_t *slots, uint64_t *groups, uint64_t *merged) {
    if (!S) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    if (slots) *slots = (uint32_t)S->slots.size();
    if (groups) *groups = S->groups;
    if (merged) *merged = S->merged;
    return MB_OK;
}

extern "C" int mb_serve_destroy(mb_server *S) {
    if (!S) return MB_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (Slot &s : S->slots) {
        cudaStreamSynchronize(s.st);
        free_slot(s);
    }
    delete S;
    return MB_OK;
}
