// Served form: continuous batching of seeding requests (the whole stage of Section 2.5 and
// Algorithm 2 per request) on one GPU.
//
// Submitting copies a request's bases into a pinned staging ring (on the caller's thread) and
// queues it.  A worker thread owns the execution slots (a stream, a seeding plan and the device
// copies of one launch group each).  Whenever a slot is free it merges every waiting request that
// still fits the slot's limits into one group, copies the group in straight from the ring, runs
// the plan and records an event; completion is handled in two asynchronous phases (the two result
// counts, then the results), so the worker never blocks on the GPU and groups on different slots
// overlap on the device.  Each request gets back exactly what mb_seed_batch + mb_locate give for
// it alone: read numbers and hit offsets are made relative to the request.
//
// Each slot runs its plan as one CUDA graph captured when the slot is made, for SLOT_READS reads:
// a group of n reads fills the offsets past its last read with its end (empty reads, which yield
// nothing), so one graph launch replaces the hundred-odd kernel launches of a plan run and the
// worker's time per group no longer bounds the request rate.
//
// Admission by free device memory: slots are created only when work is waiting and no slot is
// free, and only while the free device memory (cudaMemGetInfo) minus a reserve left to other
// users holds one more slot and the slots stay within the caller's budget; otherwise requests wait
// for a slot to free.  When free memory falls below the reserve, idle slots are released.  A group
// that yields more records or hits than its plan holds is handed to a second thread, which seeds
// its requests one by one with the allocating entry points, so the worker keeps serving.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#include "common.cuh"

namespace {

constexpr u32 SLOT_READS = 65536;
constexpr u64 SLOT_BASES = 64ull << 20;
constexpr u64 SLOT_SMEM = 2ull << 20;
constexpr u64 SLOT_HITS = 32ull << 20;
constexpr int MAX_SLOTS = 32;
constexpr u64 RING_BYTES = 1ull << 30;         // pinned staging of submitted bases
constexpr u64 RESERVE_MIN = 1ull << 30;        // free device memory left to other users (at least)
constexpr double MEM_POLL_MS = 1.0;            // how often the worker may query free memory
// A group takes as long as its longest read (Algorithm 3's steps on one read are sequential), so
// requests with reads of at least LONG_READ bases are grouped apart from the others: a request of
// short reads never waits for a long read of another request.
constexpr u64 LONG_READ = 1000;
constexpr double LONG_SLOT_SHARE = 0.5;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Pinned ring of request bases.  Positions grow monotonically (physical = pos % size); a request
// never wraps (it starts again at the beginning when it does not fit before the end).  Space is
// given back when the oldest live request is released, so requests that finish out of order wait
// for the ones before them.
struct Ring {
    u8 *base = nullptr;
    u64 size = 0, head = 0;
    std::deque<u64> beg, end;      // live allocations in order
    std::deque<bool> released;
    u64 tail() const { return beg.empty() ? head : beg.front(); }
    bool alloc(u64 bytes, u64 &pos) {
        u64 p = head;
        const u64 phys = p % size;
        if (phys + bytes > size) p += size - phys;
        if (p + bytes - tail() > size) return false;
        pos = p;
        head = p + bytes;
        beg.push_back(p);
        end.push_back(head);
        released.push_back(false);
        return true;
    }
    void release(u64 pos) {
        for (size_t i = 0; i < beg.size(); ++i)
            if (beg[i] == pos && !released[i]) {
                released[i] = true;
                break;
            }
        while (!beg.empty() && released.front()) {
            beg.pop_front();
            end.pop_front();
            released.pop_front();
        }
    }
    u8 *at(u64 pos) const { return base + pos % size; }
};

struct Request {
    u64 ticket = 0;
    u64 ring_pos = 0;        // its bases in the ring
    const u8 *seq = nullptr; // = ring.at(ring_pos)
    std::vector<u64> off;    // n_reads + 1, from 0
    u32 n_reads = 0;
    bool long_reads = false;  // holds a read of LONG_READ bases or more (grouped apart)
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
    u64 *hoff = nullptr;      // pinned
    u64 *hcnt = nullptr;      // pinned: n_smem, n_hits, the device error word
    mb_smem *hsmem = nullptr; // pinned
    u32 *hhits = nullptr;     // pinned
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t exec = nullptr;   // the plan run over SLOT_READS reads (null: launched directly)
    Phase phase = IDLE;
    std::vector<ReqP> group;
    std::vector<u32> first_read;   // first group read of each request
    u32 n_reads = 0;
    size_t dev_bytes = 0;
    double idle_since = 0;
    bool long_group = false;   // the group holds requests with long reads
};

// live servers: calls on a destroyed server are refused instead of touching freed memory
std::mutex g_live_mu;
std::unordered_set<const mb_server *> g_live;
bool alive(const mb_server *S) {
    std::lock_guard<std::mutex> g(g_live_mu);
    return S && g_live.count(S) != 0;
}

}  // namespace

struct mb_server {
    const mb_index *idx = nullptr;
    mb_opts opts{};
    int device = 0;
    u64 budget = 0;            // device bytes the slots may hold in all (0 = no cap but free memory)
    u64 reserve = RESERVE_MIN;
    size_t slot_bytes = 0;     // device bytes of one slot
    std::vector<std::unique_ptr<Slot>> slots;
    Ring ring;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ReqP> pending;
    u64 pending_short = 0;   // waiting requests without long reads
    std::unordered_map<u64, ReqP> reqs;
    std::thread worker, helper;
    std::deque<std::vector<ReqP>> outgrown;   // groups for the helper thread
    bool stop = false, helper_stop = false;
    u64 next_ticket = 1;
    // counters (mb_serve_counters)
    u64 groups = 0, merged = 0, created = 0, retired = 0, alloc_failures = 0, fallback_groups = 0, busy = 0;
    u64 long_groups = 0;
    double mem_wait_ms = 0;
    std::atomic<u64> worker_busy_us{0};   // worker thread time launching groups and handing out results
    // fault injection for tests (mb_serve_inject)
    int64_t fake_free = -1;    // free device bytes reported to admission instead of cudaMemGetInfo's
    u32 fail_next = 0;         // slot creations to fail
};

namespace {

// Offsets past a group's last read: off[i] = off[n] for n < i <= max_n, n = off[max_n + 1] (the
// count the group's copy puts after the offsets), so a plan over max_n reads sees n reads and
// max_n - n empty ones.
__global__ void k_off_tail(u64 *off, u32 max_n) {
    const u64 n = off[(u64)max_n + 1];
    if (n > max_n) return;
    const u64 end = off[n];
    for (u64 i = n + 1 + blockIdx.x * (u64)blockDim.x + threadIdx.x; i <= max_n; i += (u64)gridDim.x * blockDim.x)
        off[i] = end;
}

void free_slot(Slot &s) {
    if (s.st) cudaStreamSynchronize(s.st);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.plan) mb_plan_free(s.plan);
    if (s.dseq) cudaFree(s.dseq);
    if (s.doff) cudaFree(s.doff);
    if (s.hoff) cudaFreeHost(s.hoff);
    if (s.hcnt) cudaFreeHost(s.hcnt);
    if (s.hsmem) cudaFreeHost(s.hsmem);
    if (s.hhits) cudaFreeHost(s.hhits);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.st) cudaStreamDestroy(s.st);
    s = Slot{};
}

size_t slot_device_bytes(const mb_index *idx, const mb_opts *o) {
    u64 n = 0, prim = 0, rl = 0;
    mb_index_info(idx, &n, &prim, &rl);
    return mb_plan_workspace_bytes(o, n, SLOT_READS, SLOT_BASES, SLOT_SMEM, SLOT_HITS) + SLOT_BASES + 16 +
           (SLOT_READS + 2) * 8;
}

int make_slot(mb_server *S, Slot &s) {
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return MB_ERR_CUDA;
    }
    MB_TRY(mb_plan_create(S->idx, &S->opts, SLOT_READS, SLOT_BASES, SLOT_SMEM, SLOT_HITS, &s.plan));
    if (cudaMalloc(&s.dseq, SLOT_BASES + 16) != cudaSuccess || cudaMalloc(&s.doff, (SLOT_READS + 2) * 8) != cudaSuccess ||
        cudaMallocHost(&s.hoff, (SLOT_READS + 2) * 8) != cudaSuccess || cudaMallocHost(&s.hcnt, 32) != cudaSuccess ||
        cudaMallocHost(&s.hsmem, SLOT_SMEM * sizeof(mb_smem)) != cudaSuccess ||
        cudaMallocHost(&s.hhits, SLOT_HITS * 4) != cudaSuccess) {
        cudaGetLastError();
        return MB_ERR_NOMEM;
    }
    s.dev_bytes = mb_plan_bytes(s.plan) + SLOT_BASES + 16 + (SLOT_READS + 2) * 8;
    // the plan run as one graph: the offsets' tail, the run over SLOT_READS reads, the counts out
    // (left null when the capture fails: the worker then launches the run directly)
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        k_off_tail<<<(SLOT_READS + 255) / 256, 256, 0, s.st>>>(s.doff, SLOT_READS);
        mb_count_launch();
        const int rc = mb_plan_run(s.plan, s.dseq, s.doff, SLOT_READS, nullptr, s.st) == MB_OK &&
                               mb_plan_counts_async(s.plan, s.hcnt, s.st) == MB_OK
                           ? MB_OK
                           : MB_ERR_CUDA;
        if (cudaStreamEndCapture(s.st, &g) != cudaSuccess || rc != MB_OK ||
            cudaGraphInstantiate(&s.exec, g, 0) != cudaSuccess)
            s.exec = nullptr;
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    return MB_OK;
}

// Free device memory as admission sees it.
u64 free_device_bytes(mb_server *S) {
    if (S->fake_free >= 0) return (u64)S->fake_free;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return fr;
}

u64 slots_bytes(const mb_server *S) {
    u64 b = 0;
    for (const auto &s : S->slots) b += s->dev_bytes;
    return b;
}

// One more slot if the free device memory and the budget allow it (worker thread, lock not held).
// Returns true if a slot was added.
bool grow(mb_server *S) {
    if ((int)S->slots.size() >= MAX_SLOTS) return false;
    if (S->budget && slots_bytes(S) + S->slot_bytes > S->budget && !S->slots.empty()) return false;
    if (free_device_bytes(S) < S->reserve + S->slot_bytes) return false;
    std::unique_ptr<Slot> s(new Slot);
    int rc = MB_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);   // an allocation failure injected by mb_serve_inject
        rc = S->fail_next ? (--S->fail_next, MB_ERR_NOMEM) : MB_OK;
    }
    if (rc == MB_OK) rc = make_slot(S, *s);
    if (rc != MB_OK) {
        free_slot(*s);
        std::lock_guard<std::mutex> g(S->mu);
        ++S->alloc_failures;
        return false;
    }
    std::lock_guard<std::mutex> g(S->mu);
    S->slots.push_back(std::move(s));
    ++S->created;
    return true;
}

// Idle slots are released while free device memory is below the reserve (worker thread).
void retire(mb_server *S) {
    if (free_device_bytes(S) >= S->reserve) return;
    for (size_t i = 0; i < S->slots.size();) {
        if (S->slots[i]->phase == IDLE) {
            free_slot(*S->slots[i]);
            std::lock_guard<std::mutex> g(S->mu);
            S->slots.erase(S->slots.begin() + i);
            ++S->retired;
            if (free_device_bytes(S) >= S->reserve) return;
        } else {
            ++i;
        }
    }
}

// Merge waiting requests into the free slot s (called with the lock held): the oldest waiting
// request and, in arrival order, the later ones of its kind (long reads or not) while they fit
// the slot.  With `no_long`, the oldest waiting request without long reads leads instead (none:
// nothing is admitted).  Returns false if nothing was admitted.
bool admit(mb_server *S, Slot &s, bool no_long) {
    if (S->pending.empty()) return false;
    bool kind = S->pending.front()->long_reads, forced = false;
    if (kind && no_long) {
        if (S->pending_short == 0) return false;
        kind = false;
        forced = true;   // a request of short reads is waiting behind long ones: find it
    }
    s.group.clear();
    s.first_read.clear();
    s.long_group = kind;
    u32 nr = 0;
    u64 nb = 0;
    std::deque<ReqP> rest;
    while (!S->pending.empty()) {
        ReqP r = S->pending.front();
        S->pending.pop_front();
        const u64 b = r->off[r->n_reads];
        if (r->long_reads != kind) {
            rest.push_back(r);
            if (!forced && rest.size() >= 256) break;   // bounded look-ahead past the other kind
            continue;
        }
        if (!s.group.empty() && (nr + r->n_reads > SLOT_READS || nb + b > SLOT_BASES)) {
            S->pending.push_front(r);
            break;
        }
        s.first_read.push_back(nr);
        s.group.push_back(r);
        nr += r->n_reads;
        nb += b;
        if (!r->long_reads) --S->pending_short;
    }
    while (!rest.empty()) {   // the skipped requests go back in front, in their order
        S->pending.push_front(rest.back());
        rest.pop_back();
    }
    s.n_reads = nr;
    return !s.group.empty();
}

// Copy the group in from the ring and run it (lock not held).
int launch(mb_server *S, Slot &s) {
    u64 nb = 0;
    u32 nr = 0;
    s.hoff[0] = 0;
    // consecutive requests are usually contiguous in the ring: one copy per contiguous run
    const u8 *run = nullptr;
    u64 run_len = 0, run_dst = 0;
    for (const ReqP &r : s.group) {
        const u64 b = r->off[r->n_reads];
        for (u32 i = 0; i < r->n_reads; ++i) s.hoff[nr + i + 1] = nb + r->off[i + 1];
        if (run && run + run_len == r->seq) {
            run_len += b;
        } else {
            if (run_len) MB_CK(cudaMemcpyAsync(s.dseq + run_dst, run, run_len, cudaMemcpyHostToDevice, s.st));
            run = r->seq;
            run_len = b;
            run_dst = nb;
        }
        nb += b;
        nr += r->n_reads;
    }
    if (run_len) MB_CK(cudaMemcpyAsync(s.dseq + run_dst, run, run_len, cudaMemcpyHostToDevice, s.st));
    MB_CK(cudaMemcpyAsync(s.doff, s.hoff, (size_t)(nr + 1) * 8, cudaMemcpyHostToDevice, s.st));
    if (s.exec) {   // the group's read count after the offsets, then the captured run
        s.hoff[SLOT_READS + 1] = nr;
        MB_CK(cudaMemcpyAsync(s.doff + SLOT_READS + 1, s.hoff + SLOT_READS + 1, 8, cudaMemcpyHostToDevice, s.st));
        MB_CK(cudaGraphLaunch(s.exec, s.st));
    } else {
        MB_TRY(mb_plan_run(s.plan, s.dseq, s.doff, nr, nullptr, s.st));
        MB_TRY(mb_plan_counts_async(s.plan, s.hcnt, s.st));
    }
    MB_CK(cudaEventRecord(s.ev, s.st));
    s.phase = RUNNING;
    return MB_OK;
}

// The group's counts are on the host: copy the results back.  Returns 1 when the group outgrew
// the plan (handed to the helper thread).
int fetch(mb_server *S, Slot &s) {
    const u64 ns = s.hcnt[0], nh = s.hcnt[1];
    if (s.hcnt[2] >> 32) return MB_ERR_DEVICE_CHECK;   // (the server builds the offsets itself)
    const mb_smem *dsm;
    const u32 *dh;
    u64 ms, mh;
    mb_plan_arrays(s.plan, &dsm, &dh, &ms, &mh);
    if (ns > ms || nh > mh) {
        std::lock_guard<std::mutex> g(S->mu);
        S->outgrown.push_back(s.group);
        ++S->fallback_groups;
        S->cv.notify_all();
        s.group.clear();
        s.phase = IDLE;
        return 1;
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

// Requests done: latency, ring space back, waiters woken (lock taken here).
void complete(mb_server *S, const std::vector<ReqP> &group) {
    const double t = now_ms();
    std::lock_guard<std::mutex> g(S->mu);
    for (const ReqP &r : group) {
        r->latency_ms = t - r->t_submit;
        r->done = true;
        S->ring.release(r->ring_pos);
    }
    S->groups += 1;
    if (group.size() > 1) S->merged += group.size();
    S->cv.notify_all();
}

void finish(mb_server *S, Slot &s) {
    complete(S, s.group);
    s.group.clear();
    s.phase = IDLE;
    s.idle_since = now_ms();
}

void worker_loop(mb_server *S) {
    cudaSetDevice(S->device);
    double last_mem = -1e30, waiting_since = -1;
    for (;;) {
        bool any_busy = false, waiting = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (const auto &s : S->slots) any_busy |= s->phase != IDLE;
            if (S->stop && S->pending.empty() && !any_busy) return;
            if (S->pending.empty() && !any_busy) {
                S->cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return S->stop || !S->pending.empty(); });
                if (S->pending.empty()) {
                    lk.unlock();
                    retire(S);   // nothing to do: give memory back if others need it
                }
                continue;
            }
            waiting = !S->pending.empty();
        }
        bool progressed = false, idle_slot = false;
        for (auto &sp : S->slots) {
            Slot &s = *sp;
            if (s.phase == IDLE) {
                // long-read groups take at most LONG_SLOT_SHARE of the slots, so requests of short
                // reads always find one
                int long_busy = 0;
                for (const auto &o : S->slots) long_busy += o->phase != IDLE && o->long_group;
                const bool no_long = long_busy >= (int)(LONG_SLOT_SHARE * (double)S->slots.size()) && long_busy > 0;
                bool got;
                const double t0 = now_ms();
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    got = admit(S, s, no_long);
                    S->long_groups += got && s.long_group;
                }
                if (got) {
                    if (launch(S, s) != MB_OK) {
                        for (const ReqP &r : s.group) r->status = MB_ERR_CUDA;
                        finish(S, s);
                    }
                    progressed = true;
                    S->worker_busy_us += (u64)((now_ms() - t0) * 1000.0);
                } else {
                    idle_slot = true;
                }
            } else if (cudaEventQuery(s.ev) == cudaSuccess) {
                const double t0 = now_ms();
                if (s.phase == RUNNING) {
                    const int rc = fetch(S, s);
                    if (rc != MB_OK && rc != 1) {
                        for (const ReqP &r : s.group) r->status = rc;
                        finish(S, s);
                    }
                } else {
                    split(s);
                    finish(S, s);
                }
                progressed = true;
                S->worker_busy_us += (u64)((now_ms() - t0) * 1000.0);
            }
        }
        // work waits and every slot is busy: admission by free device memory may add a slot
        const double t = now_ms();
        if (waiting && !idle_slot && !progressed && t - last_mem >= MEM_POLL_MS) {
            last_mem = t;
            if (grow(S)) progressed = true;
            else if (waiting_since < 0) waiting_since = t;
        }
        if (progressed && waiting_since >= 0) {
            std::lock_guard<std::mutex> g(S->mu);
            S->mem_wait_ms += t - waiting_since;
            waiting_since = -1;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Groups that outgrew their plan: each request alone through the allocating entry points, on the
// helper thread's own stream (the worker is not held up).
void helper_loop(mb_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        std::vector<ReqP> group;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->helper_stop || !S->outgrown.empty(); });
            if (S->outgrown.empty()) break;
            group = std::move(S->outgrown.front());
            S->outgrown.pop_front();
        }
        for (const ReqP &r : group) {
            u64 m = 0, h = 0;
            int rc = mb_seed_batch(S->idx, r->seq, r->off.data(), r->n_reads, nullptr, &S->opts, st, nullptr, 0, &m, &h);
            if (rc != MB_OK && rc != MB_ERR_CAPACITY) {
                r->status = rc;
                continue;
            }
            r->smem.resize(m);
            rc = mb_seed_batch(S->idx, r->seq, r->off.data(), r->n_reads, nullptr, &S->opts, st, r->smem.data(), m,
                               &m, &h);
            if (rc == MB_OK) {
                r->hits.resize(h);
                rc = mb_locate(S->idx, r->smem.data(), m, &S->opts, st, r->hits.data(), h, &h);
            }
            r->status = rc;
        }
        complete(S, group);
    }
    if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" int mb_serve_create(const mb_index *idx, const mb_opts *opts, uint64_t hbm_budget, mb_server **out) {
    if (!idx || !out) return MB_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<mb_server> S(new mb_server);
    S->idx = idx;
    if (opts) S->opts = *opts;
    S->opts.flags |= MB_BATCHED;
    S->opts.flags &= ~(u32)MB_LOCATE_JOIN;   // slots stay small: no mark words per slot
    S->opts.flags &= ~(u32)MB_COUNT;
    MB_CK(cudaGetDevice(&S->device));
    S->budget = hbm_budget;
    size_t fr = 0, tot = 0;
    MB_CK(cudaMemGetInfo(&fr, &tot));
    S->reserve = tot / 50 > RESERVE_MIN ? tot / 50 : RESERVE_MIN;
    S->slot_bytes = slot_device_bytes(idx, &S->opts);
    S->ring.size = RING_BYTES;
    if (cudaMallocHost(&S->ring.base, RING_BYTES) != cudaSuccess) {
        cudaGetLastError();
        mb_set_error("mb_serve_create: cannot allocate %llu bytes of pinned staging", (unsigned long long)RING_BYTES);
        return MB_ERR_NOMEM;
    }
    mb_server *p = S.release();
    {
        std::lock_guard<std::mutex> g(g_live_mu);
        g_live.insert(p);
    }
    p->worker = std::thread(worker_loop, p);
    p->helper = std::thread(helper_loop, p);
    *out = p;
    return MB_OK;
}

extern "C" int mb_serve_submit(mb_server *S, const uint8_t *seq, const uint64_t *off, uint32_t n_reads,
                               uint64_t *ticket) {
    if (!alive(S)) {
        mb_set_error("mb_serve_submit: not a live server (destroyed?)");
        return MB_ERR_ARG;
    }
    if (!ticket || !off || (n_reads && !seq)) return MB_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->n_reads = n_reads;
    r->off.resize((size_t)n_reads + 1);
    for (u32 i = 0; i <= n_reads; ++i) r->off[i] = off[i] - off[0];
    for (u32 i = 0; i < n_reads && !r->long_reads; ++i) r->long_reads = r->off[i + 1] - r->off[i] >= LONG_READ;
    const u64 nb = r->off[n_reads];
    if (n_reads > SLOT_READS || nb > SLOT_BASES) {
        mb_set_error("mb_serve_submit: %u reads / %llu bases exceed one slot (%u / %llu)", n_reads,
                     (unsigned long long)nb, SLOT_READS, (unsigned long long)SLOT_BASES);
        return MB_ERR_ARG;
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return MB_ERR_ARG;
        if (!S->ring.alloc(nb ? nb : 1, r->ring_pos)) {
            ++S->busy;
            mb_set_error("mb_serve_submit: the staging ring is full (%llu bytes of requests outstanding)",
                         (unsigned long long)(S->ring.head - S->ring.tail()));
            return MB_ERR_BUSY;
        }
        r->seq = S->ring.at(r->ring_pos);
    }
    memcpy((void *)r->seq, seq + off[0], nb);   // the caller's thread stages the bases (pinned)
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> g(S->mu);
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    if (!r->long_reads) ++S->pending_short;
    *ticket = r->ticket;
    S->cv.notify_all();
    return MB_OK;
}

extern "C" int mb_serve_poll(mb_server *S, uint64_t ticket, int *done) {
    if (!alive(S) || !done) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return MB_ERR_ARG;
    *done = it->second->done ? 1 : 0;
    return MB_OK;
}

extern "C" int mb_serve_wait(mb_server *S, uint64_t ticket, uint32_t timeout_ms, const mb_smem **smem,
                             uint64_t *n_smem, const uint32_t **hits, uint64_t *n_hits, double *latency_ms) {
    if (!alive(S)) return MB_ERR_ARG;
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
    if (!alive(S)) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->done) return MB_ERR_ARG;
    S->reqs.erase(it);
    return MB_OK;
}

extern "C" int mb_serve_stats(mb_server *S, uint32_t *slots, uint64_t *groups, uint64_t *merged) {
    if (!alive(S)) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    if (slots) *slots = (uint32_t)S->slots.size();
    if (groups) *groups = S->groups;
    if (merged) *merged = S->merged;
    return MB_OK;
}

extern "C" int mb_serve_counters(mb_server *S, uint64_t *out, uint32_t count) {
    if (!alive(S) || (count && !out)) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    const u64 v[] = {S->slots.size(), S->groups, S->merged, S->created, S->retired, S->alloc_failures,
                     S->fallback_groups, S->busy, (u64)S->mem_wait_ms, S->slot_bytes, S->reserve, S->long_groups,
                     S->worker_busy_us.load() / 1000};
    for (u32 i = 0; i < count && i < sizeof(v) / sizeof(v[0]); ++i) out[i] = v[i];
    return MB_OK;
}

extern "C" int mb_serve_inject(mb_server *S, int64_t free_bytes, uint32_t fail_slots) {
    if (!alive(S)) return MB_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    S->fake_free = free_bytes;
    S->fail_next = fail_slots;
    S->cv.notify_all();
    return MB_OK;
}

extern "C" int mb_serve_destroy(mb_server *S) {
    {
        std::lock_guard<std::mutex> g(g_live_mu);
        if (!S || !g_live.count(S)) return MB_ERR_ARG;
        g_live.erase(S);
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->helper_stop = true;
        S->cv.notify_all();
    }
    if (S->helper.joinable()) S->helper.join();
    for (auto &s : S->slots) free_slot(*s);
    if (S->ring.base) cudaFreeHost(S->ring.base);
    delete S;
    return MB_OK;
}
