// agj_server.cpp — the served form of the probe (no counterpart in the
// paper, whose introduction motivates low-latency joins but measures none):
// a request loop over resident indexes.  Clients submit (index, host
// points) requests at any time; a scheduler thread forms a launch ("step")
// from the requests waiting whenever one of its slots is free, and runs it
// as one batched join (step_enqueue) on that slot's stream while the other
// slots' steps are in flight.  Admission is by device memory: the steps in
// flight share one device arena (a first-fit free list over a single
// allocation, sized to the HBM budget), each step taking exactly the bytes
// of its points, outputs and work space; a step that does not fit waits for
// earlier steps to return theirs.  Indexes are admitted against the free
// device memory (agj_server_add_index uploads a host-built index when it
// fits, leaving a reserve).  A slot's pinned host buffers are sized at
// creation for the largest step, so no allocation happens per request.
// Results land in the client's host buffers with submit, start and
// completion times.
//
// Also here: a Poisson load generator for the served form and the same
// arrivals served by one plain join per request, for comparison.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/agj.h"
#include "agj_handle.h"
#include "agj_index.h"
#include "agj_launch.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

uint64_t round256(uint64_t x) { return (x + 255) & ~255ull; }

constexpr uint32_t kMaxServerIndexes = 4096;

struct Request {
    uint64_t ticket = 0;
    uint32_t index_id = 0;
    const double* h_points = nullptr;
    uint64_t n = 0;
    uint32_t* h_offsets = nullptr;
    uint32_t* h_ids = nullptr;
    uint64_t ids_capacity = 0;
    bool keep = false;             // result kept until polled
    agj_request_result res{};
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // the running step's block of the device arena: [points][offsets][status][ids][work]
    char* d_mem = nullptr;
    uint64_t block = 0, block_bytes = 0;
    uint64_t off_pts = 0, off_off = 0, off_status = 0, off_ids = 0, off_work = 0, work_bytes = 0;
    char* h_mem = nullptr;         // pinned: [points][offsets][status][ids][tables]
    uint64_t h_off_pts = 0, h_off_off = 0, h_off_status = 0, h_off_ids = 0, h_off_stage = 0, stage_bytes = 0;
    bool busy = false;
    uint64_t step = 0;
    std::vector<Request*> reqs;
    std::vector<uint64_t> pofs, oofs, iofs;   // per request: point, offset and id positions
};

}  // namespace

struct agj_server {
    std::vector<const agj::Index*> X;   // capacity reserved at creation: never reallocated
    int device = 0;
    int ppt = 2, ctas = 0;
    bool host_reads = false;       // kernels read request points from host memory
    uint32_t n_slots = 4, max_req = 4096, max_refs = 1;
    uint64_t max_pts = 1ull << 20, max_ids = 0, max_pending = 1ull << 20;
    std::vector<Slot> slots;
    // device arena of the steps in flight (scheduler thread only)
    char* arena = nullptr;
    uint64_t arena_bytes = 0, in_use = 0, peak_in_use = 0, memory_waits = 0;
    std::map<uint64_t, uint64_t> free_blocks;   // offset -> size, coalesced
    uint64_t single_bound = 0;     // arena bytes a step of one largest request may need
    uint64_t reserve = 1ull << 30; // free device memory index admission leaves untouched
    uint64_t index_bytes = 0;      // device bytes of the indexes this server uploaded
    uint64_t device_bytes = 0;     // arena bytes

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> kept;
    uint64_t next_ticket = 1;
    uint64_t submitted = 0, completed = 0, rejected = 0, points = 0, steps = 0, step_req_max = 0;
    std::vector<std::pair<uint64_t, double>> latencies;   // (ticket, microseconds) of completed requests
    double busy_s = 0;
    bool stop = false;
    int fatal = AGJ_OK;
    std::thread worker;
};

namespace {

void free_slots(agj_server* S) {
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_mem) cudaFreeHost(sl.h_mem);
    }
    S->slots.clear();
    if (S->arena) cudaFree(S->arena);
    S->arena = nullptr;
}

// First-fit allocation of `bytes` (a multiple of 256) from the arena;
// returns false when no free block is large enough.
bool arena_alloc(agj_server* S, uint64_t bytes, uint64_t* off) {
    for (auto it = S->free_blocks.begin(); it != S->free_blocks.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const uint64_t rest = it->second - bytes, at = it->first + bytes;
        S->free_blocks.erase(it);
        if (rest) S->free_blocks[at] = rest;
        S->in_use += bytes;
        S->peak_in_use = std::max(S->peak_in_use, S->in_use);
        return true;
    }
    return false;
}

void arena_free(agj_server* S, uint64_t off, uint64_t bytes) {
    if (!bytes) return;
    S->in_use -= bytes;
    auto next = S->free_blocks.lower_bound(off);
    if (next != S->free_blocks.end() && off + bytes == next->first) {
        bytes += next->second;
        next = S->free_blocks.erase(next);
    }
    if (next != S->free_blocks.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += bytes;
            return;
        }
    }
    S->free_blocks[off] = bytes;
}

uint64_t largest_free(const agj_server* S) {
    uint64_t m = 0;
    for (auto& kv : S->free_blocks) m = std::max(m, kv.second);
    return m;
}

// Arena bytes of a step over requests r[0 .. m): staged points, offsets,
// status words, ids at each request's worst case, and the batched join's
// work space (exact, from the jobs' shape).
int step_arena_bytes(const agj_server* S, Request* const* r, uint32_t m, uint64_t* total, uint64_t* work) {
    std::vector<const agj::Index*> xs(m);
    std::vector<uint64_t> ns(m);
    uint64_t pts = 0, offs = 0, ids = 0;
    for (uint32_t j = 0; j < m; ++j) {
        xs[j] = S->X[r[j]->index_id];
        ns[j] = r[j]->n;
        const bool direct = S->host_reads && (reinterpret_cast<uintptr_t>(r[j]->h_points) & 15u) == 0;
        if (!direct) pts += r[j]->n * 16;
        offs += r[j]->n + 1;
        ids += r[j]->n * std::max<uint64_t>(xs[j]->stats.max_refs, 1);
    }
    uint64_t w = 0, tb = 0;
    const int rc = agj::step_bytes(xs.data(), ns.data(), m, S->ppt, &w, &tb);
    if (rc != AGJ_OK) return rc;
    *work = round256(w);
    *total = round256(pts) + round256(offs * 4) + round256((uint64_t)m * 32) + round256(ids * 4 + 4) + *work;
    return AGJ_OK;
}

// Copies a finished step's results out to its requests.
void finalize(agj_server* S, Slot& sl) {
    const uint64_t t = now_ns();
    std::vector<Request*> drop;
    for (size_t j = 0; j < sl.reqs.size(); ++j) {
        Request* r = sl.reqs[j];
        const uint64_t* st = reinterpret_cast<const uint64_t*>(sl.h_mem + sl.h_off_status) + 4 * j;
        const uint32_t* off = reinterpret_cast<const uint32_t*>(sl.h_mem + sl.h_off_off) + sl.oofs[j];
        const uint32_t* ids = reinterpret_cast<const uint32_t*>(sl.h_mem + sl.h_off_ids) + sl.iofs[j];
        const uint64_t nnz = st[0];
        int status = AGJ_OK;
        if (st[1] & 1ull) status = AGJ_ECAPACITY;
        else if (st[1] & 2ull) status = AGJ_ETIMEOUT;
        else if (st[1] & 4ull) status = AGJ_EDEVICE;
        else if (st[1] & 8ull) status = AGJ_ECAPACITY;
        if (r->h_offsets) memcpy(r->h_offsets, off, (r->n + 1) * 4);
        if (r->h_ids) {
            if (nnz > r->ids_capacity) status = status == AGJ_OK ? AGJ_ECAPACITY : status;
            else memcpy(r->h_ids, ids, nnz * 4);
        }
        r->res.status = status;
        r->res.nnz = nnz;
        r->res.t_done_ns = t;
        r->res.step = sl.step;
        if (!r->keep) drop.push_back(r);
    }
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request* r : sl.reqs) {
        r->done = true;
        ++S->completed;
        S->latencies.emplace_back(r->ticket, (r->res.t_done_ns - r->res.t_submit_ns) * 1e-3);
    }
    for (Request* r : drop) delete r;
    sl.reqs.clear();
    sl.busy = false;
    S->cv_done.notify_all();
    arena_free(S, sl.block, sl.block_bytes);       // the scheduler thread owns the arena
    sl.block_bytes = 0;
}

enum StepOutcome { kStepLaunched, kStepNothing, kStepNoMemory };

// Fails requests that never ran with status rc.
void fail_requests(agj_server* S, const std::vector<Request*>& take, int rc) {
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request* r : take) {
        r->res.status = rc;
        r->res.t_done_ns = now_ns();
        r->done = true;
        ++S->completed;
        if (!r->keep) delete r;
    }
    S->cv_done.notify_all();
}

// Forms and launches one step on a free slot from the waiting requests:
// requests are taken from the queue head while they fit a slot's buffers,
// then the step is cut back from its tail until its exact device bytes fit
// a free block of the arena (the requests cut go back to the queue head, in
// order).  kStepNoMemory: not even the head request fits now; it waits for
// a step in flight to return its block.
StepOutcome launch_step(agj_server* S, Slot& sl) {
    std::vector<Request*> take;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        uint64_t pts = 0, ids = 0;
        while (!S->pending.empty() && take.size() < S->max_req) {
            Request* r = S->pending.front();
            const uint64_t cap = r->n * std::max<uint64_t>(S->X[r->index_id]->stats.max_refs, 1);
            if (!take.empty() && (pts + r->n > S->max_pts || ids + cap > S->max_ids)) break;
            pts += r->n;
            ids += cap;
            take.push_back(r);
            S->pending.pop_front();
        }
    }
    if (take.empty()) return kStepNothing;
    // admission by device memory
    uint64_t bytes = 0, work = 0, off = 0;
    const uint64_t avail = largest_free(S);
    int rc = AGJ_OK;
    for (;;) {
        rc = step_arena_bytes(S, take.data(), (uint32_t)take.size(), &bytes, &work);
        if (rc != AGJ_OK || bytes <= avail || take.size() == 1) break;
        // cut the step to about what fits (the bytes grow with the points)
        size_t keep = (size_t)((double)take.size() * (double)avail / (double)bytes);
        keep = std::max<size_t>(1, std::min(keep, take.size() - 1));
        std::lock_guard<std::mutex> lock(S->mu);
        while (take.size() > keep) {
            S->pending.push_front(take.back());
            take.pop_back();
        }
    }
    if (rc != AGJ_OK) {
        fail_requests(S, take, rc);
        return kStepLaunched;
    }
    if (!arena_alloc(S, bytes, &off)) {
        std::lock_guard<std::mutex> lock(S->mu);
        for (auto it = take.rbegin(); it != take.rend(); ++it) S->pending.push_front(*it);
        ++S->memory_waits;
        return kStepNoMemory;
    }
    sl.block = off;
    sl.block_bytes = bytes;
    sl.d_mem = S->arena + off;
    const uint64_t t_start = now_ns();
    const uint32_t m = (uint32_t)take.size();
    // the step's block: [points][offsets][status][ids][work]
    uint64_t staged = 0, n_off = 0, n_ids = 0;
    for (Request* r : take) {
        const bool direct = S->host_reads && (reinterpret_cast<uintptr_t>(r->h_points) & 15u) == 0;
        if (!direct) staged += r->n * 16;
        n_off += r->n + 1;
        n_ids += r->n * std::max<uint64_t>(S->X[r->index_id]->stats.max_refs, 1);
    }
    sl.off_pts = 0;
    sl.off_off = round256(staged);
    sl.off_status = sl.off_off + round256(n_off * 4);
    sl.off_ids = sl.off_status + round256((uint64_t)m * 32);
    sl.off_work = sl.off_ids + round256(n_ids * 4 + 4);
    sl.work_bytes = work;
    sl.reqs = take;
    sl.pofs.resize(m);
    sl.oofs.resize(m);
    sl.iofs.resize(m);
    std::vector<const agj::Index*> xs(m);
    std::vector<uint64_t> ns(m);
    std::vector<const double*> dp(m);
    std::vector<agj_pairs> outs(m);
    uint64_t po = 0, oo = 0, io = 0;
    char* d_pts = sl.d_mem + sl.off_pts;
    for (uint32_t j = 0; j < m; ++j) {
        Request* r = take[j];
        r->res.t_start_ns = t_start;
        xs[j] = S->X[r->index_id];
        ns[j] = r->n;
        sl.pofs[j] = po;
        sl.oofs[j] = oo;
        sl.iofs[j] = io;
        const bool direct = S->host_reads && (reinterpret_cast<uintptr_t>(r->h_points) & 15u) == 0;
        if (direct) {
            dp[j] = r->h_points;                 // read by the probe over the host link
        } else {
            memcpy(sl.h_mem + sl.h_off_pts + po, r->h_points, r->n * 16);
            dp[j] = reinterpret_cast<const double*>(d_pts + po);
            po += r->n * 16;
        }
        agj_pairs& o = outs[j];
        memset(&o, 0, sizeof o);
        o.offsets = reinterpret_cast<uint32_t*>(sl.d_mem + sl.off_off) + oo;
        o.ids = reinterpret_cast<uint32_t*>(sl.d_mem + sl.off_ids) + io;
        o.ids_capacity = r->n * std::max<uint64_t>(xs[j]->stats.max_refs, 1);
        o.status = reinterpret_cast<uint64_t*>(sl.d_mem + sl.off_status) + 4 * j;
        oo += r->n + 1;
        io += o.ids_capacity;
    }
    cudaStream_t st = sl.stream;
    if (po && cudaMemcpyAsync(d_pts, sl.h_mem + sl.h_off_pts, po, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = AGJ_ECUDA;
    if (rc == AGJ_OK)
        rc = agj::step_enqueue(xs.data(), ns.data(), m, S->ppt, S->ctas, dp.data(), outs.data(),
                               sl.d_mem + sl.off_work, sl.work_bytes, sl.h_mem + sl.h_off_stage, sl.stage_bytes, st);
    if (rc == AGJ_OK &&
        (cudaMemcpyAsync(sl.h_mem + sl.h_off_off, sl.d_mem + sl.off_off, oo * 4, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(sl.h_mem + sl.h_off_status, sl.d_mem + sl.off_status, m * 32ull, cudaMemcpyDeviceToHost,
                         st) != cudaSuccess ||
         (io && cudaMemcpyAsync(sl.h_mem + sl.h_off_ids, sl.d_mem + sl.off_ids, io * 4, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess) ||
         cudaEventRecord(sl.done, st) != cudaSuccess))
        rc = AGJ_ECUDA;
    if (rc != AGJ_OK) {
        cudaGetLastError();
        // the step never ran (or its launch failed): its requests fail; the
        // block is returned once the stream has passed whatever was enqueued
        cudaStreamSynchronize(st);
        arena_free(S, sl.block, sl.block_bytes);
        sl.block_bytes = 0;
        sl.reqs.clear();
        fail_requests(S, take, rc);
        return kStepLaunched;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    sl.busy = true;
    sl.step = ++S->steps;
    S->step_req_max = std::max<uint64_t>(S->step_req_max, m);
    return kStepLaunched;
}

void run(agj_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        // retire finished steps
        for (Slot& sl : S->slots)
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) finalize(S, sl);
        bool stop;
        size_t waiting;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            stop = S->stop;
            waiting = S->pending.size();
        }
        Slot* free_slot = nullptr;
        Slot* oldest = nullptr;
        for (Slot& sl : S->slots) {
            if (!sl.busy && !free_slot) free_slot = &sl;
            if (sl.busy && (!oldest || sl.step < oldest->step)) oldest = &sl;
        }
        if (waiting && free_slot) {
            const StepOutcome o = launch_step(S, *free_slot);
            if (o != kStepNoMemory) continue;
            if (!oldest) {                 // cannot happen: submit refuses requests beyond the arena
                std::vector<Request*> head;
                {
                    std::lock_guard<std::mutex> lock(S->mu);
                    head.push_back(S->pending.front());
                    S->pending.pop_front();
                }
                fail_requests(S, head, AGJ_EBUDGET);
                continue;
            }
            // fall through: wait for the oldest step to return its memory
        }
        if (waiting && oldest) {           // every slot busy, or no memory: wait for the oldest step
            const uint64_t t0 = now_ns();
            cudaEventSynchronize(oldest->done);
            S->busy_s += (now_ns() - t0) * 1e-9;
            continue;
        }
        if (oldest) {                      // steps in flight, nothing waiting: poll both
            std::this_thread::yield();
            continue;
        }
        if (stop) break;
        std::unique_lock<std::mutex> lock(S->mu);
        S->cv_work.wait_for(lock, std::chrono::milliseconds(5), [&] { return !S->pending.empty() || S->stop; });
    }
}

double percentile(std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
}

}  // namespace

extern "C" {

int agj_server_create(const agj_index* const* indexes, uint32_t n_indexes, const agj_server_opts* opts,
                      agj_server** out) {
    if (!out || !indexes || n_indexes == 0) return AGJ_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    agj_server* S = new (std::nothrow) agj_server();
    if (!S) return AGJ_ENOMEM;
    S->device = dev;
    agj_server_opts o{};
    if (opts) o = *opts;
    if (n_indexes > kMaxServerIndexes) { delete S; return AGJ_EUNSUPPORTED; }
    S->X.reserve(kMaxServerIndexes);
    uint32_t max_refs = std::max<uint32_t>(1, o.max_refs);
    for (uint32_t k = 0; k < n_indexes; ++k) {
        if (!indexes[k] || !indexes[k]->X.d_blob || indexes[k]->X.device != dev) { delete S; return AGJ_EINVAL; }
        S->X.push_back(&indexes[k]->X);
        max_refs = std::max<uint32_t>(max_refs, indexes[k]->X.stats.max_refs);
    }
    S->max_refs = max_refs;
    if (o.hbm_reserve_bytes) S->reserve = o.hbm_reserve_bytes;
    if (o.n_slots) S->n_slots = o.n_slots;
    if (o.max_step_requests) S->max_req = o.max_step_requests;
    if (o.max_step_points) S->max_pts = o.max_step_points;
    if (o.max_pending) S->max_pending = o.max_pending;
    S->ppt = o.points_per_lane ? (int)o.points_per_lane : 2;
    S->ctas = (int)o.ctas_per_sm;
    {
        int pageable = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
            cudaGetLastError();
            pageable = 0;
        }
        S->host_reads = pageable == 1 && !(o.flags & AGJ_SERVER_STAGE_POINTS);
    }
    if (S->n_slots > 64 || S->max_req > 65535 || S->max_pts >= (1ull << 31)) { delete S; return AGJ_EINVAL; }
    S->max_ids = S->max_pts * max_refs;
    // bounds of the largest step (any index, up to max_step_points points
    // in max_step_requests requests) and of the largest single request
    uint64_t work = 0, stage = 0, work1 = 0, stage1 = 0;
    {
        uint32_t mcr = 1;
        uint64_t all_polys = 0, max_polys = 0;
        for (auto* x : S->X) {
            mcr = std::max<uint32_t>(mcr, x->stats.max_cand_refs);
            if (x->mode != AGJ_EXACT) continue;
            all_polys += x->n_polys;
            max_polys = std::max<uint64_t>(max_polys, x->n_polys);
        }
        int rc = agj::step_bound(S->max_pts, S->max_req, S->ppt, mcr, all_polys, true, &work, &stage);
        if (rc == AGJ_OK) rc = agj::step_bound(S->max_pts, 1, S->ppt, mcr, max_polys, true, &work1, &stage1);
        if (rc != AGJ_OK) { delete S; return rc; }
    }
    const uint64_t pts_bytes = round256(S->max_pts * 16 + (uint64_t)S->max_req * 16);
    const uint64_t off_bytes = round256((S->max_pts + S->max_req) * 4);
    const uint64_t st_bytes = round256((uint64_t)S->max_req * 32);
    const uint64_t ids_bytes = round256(S->max_ids * 4 + 4);
    const uint64_t per_step = pts_bytes + off_bytes + st_bytes + ids_bytes + round256(work);
    S->single_bound = round256(S->max_pts * 16) + round256((S->max_pts + 1) * 4) + 256 +
                      round256(S->max_pts * max_refs * 4 + 4) + round256(work1);
    // the arena: the budget, else n_slots largest steps, within the free
    // device memory less the reserve
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); delete S; return AGJ_ECUDA; }
        const uint64_t avail = free_b > S->reserve ? free_b - S->reserve : 0;
        uint64_t want = o.hbm_budget_bytes ? o.hbm_budget_bytes : per_step * S->n_slots;
        if (want > avail) {
            if (o.hbm_budget_bytes) { delete S; return AGJ_EBUDGET; }
            want = avail;
        }
        S->arena_bytes = want & ~255ull;
        if (S->arena_bytes < 256) { delete S; return AGJ_EBUDGET; }
    }
    if (cudaMalloc(&S->arena, S->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return AGJ_ENOMEM;
    }
    S->free_blocks[0] = S->arena_bytes;
    S->device_bytes = S->arena_bytes;
    S->slots.resize(S->n_slots);
    for (Slot& sl : S->slots) {
        sl.h_off_pts = 0;
        sl.h_off_off = pts_bytes;
        sl.h_off_status = sl.h_off_off + off_bytes;
        sl.h_off_ids = sl.h_off_status + st_bytes;
        sl.h_off_stage = sl.h_off_ids + ids_bytes;
        sl.stage_bytes = round256(stage);
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_mem, sl.h_off_stage + sl.stage_bytes) != cudaSuccess) {
            cudaGetLastError();
            free_slots(S);
            delete S;
            return AGJ_ENOMEM;
        }
    }
    S->worker = std::thread(run, S);
    *out = S;
    return AGJ_OK;
}

int agj_server_submit(agj_server* S, uint32_t index_id, const double* h_points, uint64_t n, uint32_t* h_offsets,
                      uint32_t* h_ids, uint64_t ids_capacity, uint64_t* ticket) {
    if (!S || (n && !h_points) || (h_ids && !h_offsets)) return AGJ_EINVAL;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (index_id >= S->X.size()) return AGJ_EINVAL;
    }
    if (n > S->max_pts) return AGJ_ECAPACITY;
    Request* r = new (std::nothrow) Request();
    if (!r) return AGJ_ENOMEM;
    r->index_id = index_id;
    r->h_points = h_points;
    r->n = n;
    uint64_t single_bound;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        single_bound = S->single_bound;
    }
    if (single_bound > S->arena_bytes) {
        // a small arena: this request alone must fit it
        uint64_t bytes = 0, work = 0;
        const int rc = step_arena_bytes(S, &r, 1, &bytes, &work);
        if (rc != AGJ_OK || bytes > S->arena_bytes) {
            delete r;
            return rc != AGJ_OK ? rc : AGJ_EBUDGET;
        }
    }
    r->index_id = index_id;
    r->h_points = h_points;
    r->n = n;
    r->h_offsets = h_offsets;
    r->h_ids = h_ids;
    r->ids_capacity = ids_capacity;
    r->keep = h_offsets != nullptr;
    r->res.t_submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop || S->fatal != AGJ_OK) { delete r; return S->fatal != AGJ_OK ? S->fatal : AGJ_EINVAL; }
        if (S->pending.size() >= S->max_pending) {
            ++S->rejected;
            delete r;
            return AGJ_EBUSY;
        }
        r->ticket = S->next_ticket++;
        if (r->keep) S->kept[r->ticket] = r;
        S->pending.push_back(r);
        ++S->submitted;
        S->points += n;
        if (ticket) *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return AGJ_OK;
}

int agj_server_add_index(agj_server* S, agj_index* index, uint32_t* index_id) {
    if (!S || !index || !index_id) return AGJ_EINVAL;
    agj::Index& X = index->X;
    if (X.stats.max_refs > S->max_refs) return AGJ_ECAPACITY;     // the slots' pinned id buffers
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->X.size() >= kMaxServerIndexes) return AGJ_EUNSUPPORTED;
    }
    if (cudaSetDevice(S->device) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    if (!X.d_blob) {
        // admission by free device memory: the index's blob must fit what is
        // free beyond the reserve
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
        const uint64_t need = agj::index_device_bytes(X);
        if (free_b <= S->reserve || free_b - S->reserve < need) return AGJ_EBUDGET;
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
        const int rc = agj::upload_index(&X, st);
        cudaStreamDestroy(st);
        if (rc != AGJ_OK) return rc;
        std::lock_guard<std::mutex> lock(S->mu);
        S->index_bytes += X.blob_bytes;
    } else if (X.device != S->device) {
        return AGJ_EINVAL;
    }
    // the bound of one request of this index (a small arena checks requests at submit)
    uint64_t work1 = 0, stage1 = 0;
    const int rc = agj::step_bound(S->max_pts, 1, S->ppt, std::max<uint32_t>(1, X.stats.max_cand_refs),
                                   X.mode == AGJ_EXACT ? X.n_polys : 0, X.mode == AGJ_EXACT, &work1, &stage1);
    if (rc != AGJ_OK) return rc;
    const uint64_t one = round256(S->max_pts * 16) + round256((S->max_pts + 1) * 4) + 256 +
                         round256(S->max_pts * std::max<uint64_t>(X.stats.max_refs, 1) * 4 + 4) + round256(work1);
    std::lock_guard<std::mutex> lock(S->mu);
    S->single_bound = std::max(S->single_bound, one);
    S->X.push_back(&X);
    *index_id = (uint32_t)(S->X.size() - 1);
    return AGJ_OK;
}

int agj_server_poll(agj_server* S, uint64_t ticket, int wait, agj_request_result* out) {
    if (!S) return AGJ_EINVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->kept.find(ticket);
    if (it == S->kept.end()) return AGJ_EINVAL;
    Request* r = it->second;
    if (!r->done) {
        if (!wait) return AGJ_EBUSY;
        S->cv_done.wait(lock, [&] { return r->done; });
    }
    if (out) *out = r->res;
    S->kept.erase(it);
    delete r;
    return AGJ_OK;
}

int agj_server_drain(agj_server* S) {
    if (!S) return AGJ_EINVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    S->cv_done.wait(lock, [&] { return S->completed == S->submitted; });
    return AGJ_OK;
}

int agj_server_get_stats(agj_server* S, int reset, agj_server_stats* out) {
    if (!S || !out) return AGJ_EINVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->points = S->points;
    out->steps = S->steps;
    out->step_requests_max = S->step_req_max;
    out->n_slots = S->n_slots;
    out->host_reads = S->host_reads ? 1u : 0u;
    out->device_bytes = S->device_bytes;
    out->memory_waits = S->memory_waits;
    out->peak_bytes_in_use = S->peak_in_use;
    out->index_bytes = S->index_bytes;
    out->n_indexes = (uint32_t)S->X.size();
    std::vector<double> v;
    v.reserve(S->latencies.size());
    double sum = 0, mx = 0;
    for (auto& e : S->latencies) {
        v.push_back(e.second);
        sum += e.second;
        mx = std::max(mx, e.second);
    }
    out->mean_us = v.empty() ? 0.0 : sum / (double)v.size();
    out->max_us = mx;
    out->p50_us = percentile(v, 0.50);
    out->p99_us = percentile(v, 0.99);
    if (reset) {
        S->memory_waits = 0;
        S->latencies.clear();
        S->submitted -= S->completed;
        S->completed = 0;
        S->rejected = 0;
        S->points = 0;
        S->steps = 0;
        S->step_req_max = 0;
    }
    return AGJ_OK;
}

void agj_server_destroy(agj_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    agj_server_drain(S);
    if (S->worker.joinable()) S->worker.join();
    free_slots(S);
    for (auto& kv : S->kept) delete kv.second;
    delete S;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// load generation
// ---------------------------------------------------------------------------

namespace {

struct Arrival {
    double t;          // seconds after the start
    uint32_t index_id;
    const double* pts;
    uint64_t n;
};

// Poisson arrivals at spec->rate; sizes k in 1..max_points with P(k)
// proportional to k^-alpha (inverse-CDF table); a uniformly chosen set; the
// exact index with probability exact_fraction; points a random contiguous
// slice of the set's pool.
int make_arrivals(const agj_load_spec* sp, std::vector<Arrival>* out) {
    if (!sp || sp->rate <= 0 || sp->n_sets == 0 || !sp->approx_index || !sp->pools || !sp->pool_points ||
        sp->max_points == 0)
        return AGJ_EINVAL;
    for (uint32_t s = 0; s < sp->n_sets; ++s)
        if (!sp->pools[s] || sp->pool_points[s] < sp->max_points) return AGJ_EINVAL;
    std::mt19937_64 rng(sp->seed);
    std::exponential_distribution<double> gap(sp->rate);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    std::vector<double> cdf(sp->max_points);
    double acc = 0;
    for (uint32_t k = 1; k <= sp->max_points; ++k) {
        acc += std::pow((double)k, -sp->zipf_alpha);
        cdf[k - 1] = acc;
    }
    for (double& c : cdf) c /= acc;
    out->resize(sp->n_requests);
    double t = 0;
    for (uint64_t i = 0; i < sp->n_requests; ++i) {
        t += gap(rng);
        Arrival& a = (*out)[i];
        a.t = t;
        a.n = (uint64_t)(std::lower_bound(cdf.begin(), cdf.end(), u01(rng)) - cdf.begin()) + 1;
        a.n = std::min<uint64_t>(a.n, sp->max_points);
        const uint32_t set = (uint32_t)(u01(rng) * sp->n_sets) % sp->n_sets;
        const bool exact = sp->exact_index && sp->exact_index[set] != 0xFFFFFFFFu && u01(rng) < sp->exact_fraction;
        a.index_id = exact ? sp->exact_index[set] : sp->approx_index[set];
        const uint64_t start = (uint64_t)(u01(rng) * (double)(sp->pool_points[set] - a.n + 1));
        a.pts = sp->pools[set] + 2 * std::min(start, sp->pool_points[set] - a.n);
    }
    return AGJ_OK;
}

void wait_until(Clock::time_point t) {
    for (;;) {
        const auto d = t - Clock::now();
        if (d <= std::chrono::nanoseconds(0)) return;
        if (d > std::chrono::microseconds(200)) std::this_thread::sleep_for(d - std::chrono::microseconds(100));
    }
}

void summarize(std::vector<double>& lat, uint64_t requests, uint64_t points, double seconds, double offered,
               uint64_t rejected, agj_load_result* out) {
    memset(out, 0, sizeof *out);
    out->requests = requests;
    out->points = points;
    out->seconds = seconds;
    out->offered_rate = offered;
    out->achieved_rate = seconds > 0 ? (double)requests / seconds : 0.0;
    out->points_per_s = seconds > 0 ? (double)points / seconds : 0.0;
    out->rejected = rejected;
    double sum = 0, mx = 0;
    for (double x : lat) {
        sum += x;
        mx = std::max(mx, x);
    }
    out->mean_us = lat.empty() ? 0.0 : sum / (double)lat.size();
    out->max_us = mx;
    out->p50_us = percentile(lat, 0.50);
    out->p99_us = percentile(lat, 0.99);
}

}  // namespace

extern "C" {

int agj_server_load(agj_server* S, const agj_load_spec* sp, agj_load_result* out) {
    if (!S || !out) return AGJ_EINVAL;
    std::vector<Arrival> arr;
    int rc = make_arrivals(sp, &arr);
    if (rc != AGJ_OK) return rc;
    for (const Arrival& a : arr)
        if (a.index_id >= S->X.size()) return AGJ_EINVAL;
    agj_server_drain(S);
    agj_server_stats st;
    agj_server_get_stats(S, 1, &st);      // latencies from here on
    uint64_t first = 0, rejected = 0, points = 0, last_t = 0;
    const auto t0 = Clock::now();
    for (uint64_t i = 0; i < arr.size(); ++i) {
        wait_until(t0 + std::chrono::nanoseconds((int64_t)(arr[i].t * 1e9)));
        uint64_t ticket = 0;
        rc = agj_server_submit(S, arr[i].index_id, arr[i].pts, arr[i].n, nullptr, nullptr, 0, &ticket);
        if (rc == AGJ_EBUSY) { ++rejected; continue; }
        if (rc != AGJ_OK) return rc;
        if (i == sp->warmup_requests) first = ticket;
        if (i >= sp->warmup_requests) points += arr[i].n;
        last_t = ticket;
    }
    agj_server_drain(S);
    const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
    std::vector<double> lat;
    uint64_t requests = 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        for (auto& e : S->latencies)
            if (first && e.first >= first && e.first <= last_t) {
                lat.push_back(e.second);
                ++requests;
            }
    }
    // throughput over the measured part: its requests and points over the
    // time from the first measured arrival to the end
    const double t_first = sp->warmup_requests < arr.size() ? arr[sp->warmup_requests].t : 0.0;
    summarize(lat, requests, points, secs - t_first, sp->rate, rejected, out);
    return AGJ_OK;
}

int agj_plain_load(const agj_index* const* indexes, uint32_t n_indexes, const agj_load_spec* sp,
                   agj_load_result* out) {
    if (!indexes || n_indexes == 0 || !out) return AGJ_EINVAL;
    std::vector<Arrival> arr;
    int rc = make_arrivals(sp, &arr);
    if (rc != AGJ_OK) return rc;
    uint32_t max_refs = 1;
    for (uint32_t k = 0; k < n_indexes; ++k) {
        if (!indexes[k] || !indexes[k]->X.d_blob) return AGJ_EINVAL;
        max_refs = std::max<uint32_t>(max_refs, indexes[k]->X.stats.max_refs);
    }
    for (const Arrival& a : arr)
        if (a.index_id >= n_indexes) return AGJ_EINVAL;
    // one work space for the largest request over every index
    uint64_t scratch = 0;
    for (uint32_t k = 0; k < n_indexes; ++k) {
        agj_requirements r;
        agj::join_requirements(indexes[k]->X, sp->max_points, &r);
        scratch = std::max(scratch, r.scratch_bytes);
    }
    cudaStream_t s = nullptr;
    char* d = nullptr;
    char* h = nullptr;
    const uint64_t np = sp->max_points;
    const uint64_t d_bytes = round256(np * 16) + round256((np + 1) * 4) + round256(np * max_refs * 4) + 256 +
                             round256(scratch);
    const uint64_t h_bytes = round256(np * 16) + round256((np + 1) * 4) + round256(np * max_refs * 4);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaMalloc(&d, d_bytes) != cudaSuccess ||
        cudaMallocHost(&h, h_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (d) cudaFree(d);
        if (s) cudaStreamDestroy(s);
        return AGJ_ENOMEM;
    }
    double* d_pts = reinterpret_cast<double*>(d);
    agj_pairs o{};
    o.offsets = reinterpret_cast<uint32_t*>(d + round256(np * 16));
    o.ids = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(o.offsets) + round256((np + 1) * 4));
    o.ids_capacity = np * max_refs;
    o.status = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(o.ids) + round256(np * max_refs * 4));
    o.scratch = reinterpret_cast<char*>(o.status) + 256;
    o.scratch_bytes = scratch;
    char* h_pts = h;
    uint32_t* h_off = reinterpret_cast<uint32_t*>(h + round256(np * 16));
    uint32_t* h_ids = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(h_off) + round256((np + 1) * 4));
    std::vector<double> lat;
    uint64_t points = 0;
    const auto t0 = Clock::now();
    for (uint64_t i = 0; i < arr.size() && rc == AGJ_OK; ++i) {
        const Arrival& a = arr[i];
        const auto t_arr = t0 + std::chrono::nanoseconds((int64_t)(a.t * 1e9));
        wait_until(t_arr);
        // the plain path of a host request: stage, copy in, join, copy out
        memcpy(h_pts, a.pts, a.n * 16);
        rc = agj_join_host(indexes[a.index_id], reinterpret_cast<const double*>(h_pts), a.n, d_pts, &o, h_off, h_ids,
                           o.ids_capacity, nullptr, s);
        if (i >= sp->warmup_requests) {
            lat.push_back(std::chrono::duration<double, std::micro>(Clock::now() - t_arr).count());
            points += a.n;
        }
    }
    const double t_first = sp->warmup_requests < arr.size() ? arr[sp->warmup_requests].t : 0.0;
    const double secs = std::chrono::duration<double>(Clock::now() - t0).count() - t_first;
    cudaStreamSynchronize(s);
    cudaFreeHost(h);
    cudaFree(d);
    cudaStreamDestroy(s);
    if (rc != AGJ_OK) return rc;
    summarize(lat, lat.size(), points, secs, sp->rate, 0, out);
    return AGJ_OK;
}

}  // extern "C"
