// agj_batch.cu — the batched form of the probe (no counterpart in the paper):
// many (index, point batch) jobs of uneven sizes joined by one launch
// sequence.  The jobs' warp tiles are laid end to end in one tile space
// (each job padded to whole CTAs, so a CTA's tiles share a job), their exact
// indexes' polygons in one polygon space (one range per distinct index), and
// the probe, refine, scan and emit kernels run once over all of it.
//
// Two users share the code here:
//   * Batch (agj_batch_*): a plan for fixed (index, point count) jobs, with
//     its own device memory and a CUDA graph captured once; a run uploads
//     the job descriptors (only when a pointer changed) and replays the graph;
//   * step_enqueue (the served form): one launch for a set of jobs formed on
//     the fly, into a caller's device work space, with its tables staged
//     through a caller's pinned buffer.
//
// Each job computes what the plain join computes for it, bit for bit: the
// same probe per point, the same candidate set and refine test, the same
// CSR (offsets of a job are differences of prefixes of its own tiles).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "agj_index.h"
#include "agj_join.cuh"
#include "agj_launch.h"
#include "agj_probe.cuh"

namespace agj {

constexpr uint32_t kMaxBatchJobs = 65535;   // jobs are named by 16-bit ids per tile

// Clears each job's status and diagnostics and writes offsets[0] = 0 for
// empty jobs (their tiles do not exist, so no emit writes it).
__global__ void __launch_bounds__(256) k_jobs_init(const JobDesc* __restrict__ jobs, uint32_t m) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const JobDesc& J = jobs[j];
        J.status[0] = 0;
        J.status[1] = 0;
        J.status[2] = 0;
        J.status[3] = 0;
        J.counters[0] = 0;
        J.counters[1] = 0;
        if (J.n == 0) J.offsets[0] = 0;
    }
}

// The shape of one batched launch: where each job sits in the tile and
// polygon spaces, and the device memory it needs, as offsets from a base:
//   [job descriptors][job of each tile u16]   <- the tables a launch uploads
//   [job bases u32][per-job counters 2 x u64][join work space]
// The approximate jobs' tiles come first (tiles 0 .. Ta - 1), the exact
// jobs' after them, each in the callers' order, so each mode's probe and emit
// run as their own launch, compiled for that mode.
struct Shape {
    uint32_t m = 0;
    int ppt = 2;
    uint64_t T = 0, P = 0, Ta = 0;
    std::vector<uint64_t> tile0;   // m: first tile of each job
    std::vector<uint64_t> tile1;   // m: end of each job's tiles
    std::vector<uint32_t> poly0;   // m
    JoinLayout L;
    uint64_t off_jobs = 0, off_tile_job = 0, table_bytes = 0;
    uint64_t off_job_base = 0, off_counters = 0, off_scratch = 0, bytes = 0;
};

namespace {

int make_shape(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int dev, Shape* S) {
    if (m > kMaxBatchJobs) return AGJ_EUNSUPPORTED;
    S->m = m;
    S->ppt = ppt;
    S->tile0.assign(m, 0);
    S->tile1.assign(m, 0);
    S->poly0.assign(m, 0);
    uint64_t T = 0, P = 0;
    uint32_t mcr = 1;    // most candidate references of a point over the exact jobs
    bool any_exact = false;
    std::vector<std::pair<const Index*, uint32_t>> poly_base;   // exact indexes and their polygon ranges
    for (uint32_t j = 0; j < m; ++j) {
        const Index* x = X[j];
        if (!x || !x->d_blob || x->device != dev || n[j] >= 0xFFFFFFFFull) return AGJ_EINVAL;
        if (n[j] * std::max<uint64_t>(x->stats.max_refs, 1) >= 0xFFFFFFFFull) return AGJ_ECAPACITY;
    }
    // tiles: the approximate jobs, then the exact ones; whole CTAs per job,
    // so a CTA's tiles share one job
    for (int exact = 0; exact < 2; ++exact) {
        if (exact) S->Ta = T;
        for (uint32_t j = 0; j < m; ++j) {
            if ((X[j]->mode == AGJ_EXACT) != (exact == 1)) continue;
            S->tile0[j] = T;
            T += (n[j] + 32 * ppt - 1) / (32 * ppt);
            T = (T + kWarpsPerBlock - 1) / kWarpsPerBlock * kWarpsPerBlock;
            S->tile1[j] = T;
        }
    }
    for (uint32_t j = 0; j < m; ++j) {
        const Index* x = X[j];
        uint32_t pb = 0;
        if (x->mode == AGJ_EXACT) {
            any_exact = true;
            mcr = std::max<uint32_t>(mcr, x->stats.max_cand_refs);
            auto it = std::find_if(poly_base.begin(), poly_base.end(), [&](const auto& e) { return e.first == x; });
            if (it == poly_base.end()) {
                poly_base.emplace_back(x, (uint32_t)P);
                pb = (uint32_t)P;
                P += x->n_polys;
            } else {
                pb = it->second;
            }
        }
        S->poly0[j] = pb;
    }
    const uint32_t slots = 32u * (uint32_t)ppt * mcr;
    if (P >= 0xFFFFFFFFull || T * 32 * ppt >= 0xFFFFFFFFull || (any_exact && T * slots >= 0xFFFFFFFFull))
        return AGJ_ECAPACITY;   // 32-bit point, polygon and queue indices
    S->T = T;
    S->P = P;
    S->L = join_layout(T * 32 * ppt, T, any_exact, any_exact ? slots : 0u, P);
    uint64_t o = 0;
    S->off_jobs = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * sizeof(JobDesc));
    S->off_tile_job = o; o += align256(T * 2 + 2);
    S->table_bytes = o;
    S->off_job_base = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * 4);
    S->off_counters = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * 16);
    S->off_scratch = o; o += S->L.total;
    S->bytes = o;
    return AGJ_OK;
}

void fill_tile_job(const Shape& S, uint16_t* tile_job) {
    for (uint32_t j = 0; j < S.m; ++j)
        std::fill(tile_job + S.tile0[j], tile_job + S.tile1[j], (uint16_t)j);
}

// Job descriptors of one launch; counters: the per-job diagnostic words in
// device memory (used where the caller passes no work space).
int fill_jobs(const Shape& S, const Index* const* X, const uint64_t* n, const double* const* d_points,
              agj_pairs* outs, uint64_t* counters, JobDesc* jobs) {
    for (uint32_t j = 0; j < S.m; ++j) {
        agj_pairs* o = &outs[j];
        const Index& x = *X[j];
        if (!o->offsets || !o->status || (n[j] && !d_points[j])) return AGJ_EINVAL;
        if ((reinterpret_cast<uintptr_t>(d_points[j]) & 15u) != 0) return AGJ_EINVAL;
        const uint64_t need = n[j] * std::max<uint64_t>(x.stats.max_refs, 1);
        if (o->ids_capacity < need || (need && !o->ids)) return AGJ_ECAPACITY;
        // diagnostics go where the plain join puts them when the caller
        // passes a work space
        uint64_t* c = (o->scratch && o->scratch_bytes >= 32) ? static_cast<uint64_t*>(o->scratch) + 2 : counters + 2 * j;
        JobDesc J = make_job(x, d_points[j], n[j], o, c);
        J.tile0 = S.tile0[j];
        J.poly0 = S.poly0[j];
        memcpy(&jobs[j], &J, sizeof J);
    }
    return AGJ_OK;
}

// An auxiliary stream and fork/join events: where the two modes' chains of a
// large mixed launch may run side by side (a captured graph's branches).
struct Aux {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

template <int PPT>
cudaError_t enqueue_kernels(const Shape& S, char* base, int ctas_per_sm, cudaStream_t s, const Aux* aux) {
    ManyJobs src;
    src.d = reinterpret_cast<const JobDesc*>(base + S.off_jobs);
    src.tile_job = reinterpret_cast<const uint16_t*>(base + S.off_tile_job);
    src.base = reinterpret_cast<const uint32_t*>(base + S.off_job_base);
    src.m = S.m;
    src.t0 = 0;
    src.ta = S.Ta;
    k_jobs_init<<<(S.m + 255) / 256, 256, 0, s>>>(src.d, S.m);
    JoinLaunch G;
    G.sms = sm_count();
    // per mode: one warp per tile, or persistent grids (the emit is short and
    // latency-bound: a full-occupancy grid)
    auto grids = [&](uint64_t tiles, int* probe, int* emit) {
        const uint64_t need = std::max<uint64_t>(1, (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
        *probe = (int)(ctas_per_sm == 0 ? need : std::min<uint64_t>(need, (uint64_t)G.sms * ctas_per_sm));
        *emit = (int)(ctas_per_sm == 0 ? need : std::min<uint64_t>(need, (uint64_t)G.sms * 8));
    };
    G.persistent = ctas_per_sm != 0;
    G.pip_grid = G.sms * AGJ_PIP_MIN_BLOCKS;
    G.tile_job = src.tile_job;
    G.job_base = reinterpret_cast<uint32_t*>(base + S.off_job_base);
    char* sc = base + S.off_scratch;
    // One mode: that mode's kernels.  Both, over many tiles (16 waves and
    // more, ~6e6 points): each mode's chain of kernels on its own tiles (the
    // approximate probe at 6 CTAs per SM, no per-job mode branches, the
    // chains side by side where an auxiliary stream is given); over fewer (a
    // served step) the extra launches cost more than they save, so one
    // launch reads each job's mode.
    const uint64_t split_min = (uint64_t)G.sms * AGJ_PROBE_MIN_BLOCKS * kWarpsPerBlock * 16;
    if (S.Ta == S.T || S.Ta == 0 || S.T < split_min) {
        grids(S.T, &G.probe_grid, &G.emit_grid);
        if (S.Ta == S.T) return enqueue_join<PPT, ManyJobs, kModeApprox>(src, S.L, sc, G, nullptr, 0, s, nullptr);
        if (S.Ta == 0) return enqueue_join<PPT, ManyJobs, kModeExact>(src, S.L, sc, G, nullptr, 0, s, nullptr);
        return enqueue_join<PPT, ManyJobs, kModeAny>(src, S.L, sc, G, nullptr, 0, s, nullptr);
    }
    grids(S.Ta, &G.probe_grid_a, &G.emit_grid_a);
    grids(S.T - S.Ta, &G.probe_grid, &G.emit_grid);
    return enqueue_join_split<PPT>(src, S.L, sc, G, s, aux ? aux->stream : nullptr, aux ? aux->fork : nullptr,
                                   aux ? aux->join : nullptr);
}

cudaError_t enqueue(const Shape& S, char* base, int ctas_per_sm, cudaStream_t s, const Aux* aux = nullptr) {
    switch (S.ppt) {
        case 1: return enqueue_kernels<1>(S, base, ctas_per_sm, s, aux);
        case 4: return enqueue_kernels<4>(S, base, ctas_per_sm, s, aux);
        default: return enqueue_kernels<2>(S, base, ctas_per_sm, s, aux);
    }
}

int check_options(int* ppt, int ctas_per_sm) {
    if (*ppt == 0) *ppt = 2;
    if (*ppt != 1 && *ppt != 2 && *ppt != 4) return AGJ_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 8) return AGJ_EINVAL;
    return AGJ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------

struct Batch {
    Shape S;
    int ctas_per_sm = 0;                // 0: one warp per tile, else persistent grids
    int device = 0;
    std::vector<const Index*> X;
    std::vector<uint64_t> n;
    char* d_mem = nullptr;
    JobDesc* h_jobs = nullptr;          // pinned staging of the descriptors
    std::vector<JobDesc> last;          // descriptors of the last upload
    bool uploaded = false;
    cudaEvent_t upload_done = nullptr;
    cudaStream_t cap_stream = nullptr;
    Aux cap_aux;                        // second branch of the captured graph
    cudaGraphExec_t exec = nullptr;
};

void batch_free(Batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    if (B->cap_aux.stream) cudaStreamDestroy(B->cap_aux.stream);
    if (B->cap_aux.fork) cudaEventDestroy(B->cap_aux.fork);
    if (B->cap_aux.join) cudaEventDestroy(B->cap_aux.join);
    if (B->upload_done) cudaEventDestroy(B->upload_done);
    if (B->h_jobs) cudaFreeHost(B->h_jobs);
    if (B->d_mem) cudaFree(B->d_mem);
    delete B;
}

int batch_create(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int ctas_per_sm, bool use_graph,
                 Batch** out) {
    if (!out || (m && (!X || !n))) return AGJ_EINVAL;
    *out = nullptr;
    int rc = check_options(&ppt, ctas_per_sm);
    if (rc != AGJ_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    Batch* B = new (std::nothrow) Batch();
    if (!B) return AGJ_ENOMEM;
    rc = make_shape(X, n, m, ppt, dev, &B->S);
    if (rc != AGJ_OK) { delete B; return rc; }
    B->ctas_per_sm = ctas_per_sm;
    B->device = dev;
    B->X.assign(X, X + m);
    B->n.assign(n, n + m);
    const Shape& S = B->S;
    if (cudaMalloc(&B->d_mem, S.bytes) != cudaSuccess) { cudaGetLastError(); B->d_mem = nullptr; batch_free(B); return AGJ_ENOMEM; }
    if (cudaMallocHost(&B->h_jobs, (uint64_t)std::max<uint32_t>(m, 1) * sizeof(JobDesc)) != cudaSuccess) {
        cudaGetLastError();
        B->h_jobs = nullptr;
        batch_free(B);
        return AGJ_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&B->upload_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        batch_free(B);
        return AGJ_ECUDA;
    }
    // the tile-to-job table never changes for a plan
    std::vector<uint16_t> tile_job(S.T);
    fill_tile_job(S, tile_job.data());
    cudaError_t e = cudaSuccess;
    if (S.T)
        e = cudaMemcpyAsync(B->d_mem + S.off_tile_job, tile_job.data(), S.T * 2, cudaMemcpyHostToDevice, B->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->cap_stream);
    if (e != cudaSuccess) { cudaGetLastError(); batch_free(B); return AGJ_ECUDA; }
    if (use_graph && m) {
        if (cudaStreamCreateWithFlags(&B->cap_aux.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->cap_aux.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->cap_aux.join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            batch_free(B);
            return AGJ_ECUDA;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(S, B->d_mem, ctas_per_sm, B->cap_stream, &B->cap_aux);
            e = cudaStreamEndCapture(B->cap_stream, &g);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) { cudaGetLastError(); B->exec = nullptr; batch_free(B); return AGJ_ECUDA; }
    }
    *out = B;
    return AGJ_OK;
}

uint64_t batch_device_bytes(const Batch* B) { return B ? B->S.bytes : 0; }

int batch_run(Batch* B, const double* const* d_points, cudaStream_t s, agj_pairs* outs) {
    if (!B) return AGJ_EINVAL;
    const Shape& S = B->S;
    if (S.m == 0) return AGJ_OK;
    if (!d_points || !outs) return AGJ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != B->device) { cudaGetLastError(); return AGJ_EINVAL; }
    std::vector<JobDesc> jobs(S.m);
    const int rc = fill_jobs(S, B->X.data(), B->n.data(), d_points, outs,
                             reinterpret_cast<uint64_t*>(B->d_mem + S.off_counters), jobs.data());
    if (rc != AGJ_OK) return rc;
    const bool same = B->uploaded && memcmp(jobs.data(), B->last.data(), jobs.size() * sizeof(JobDesc)) == 0;
    if (!same) {
        // the staging buffer may still feed the previous upload
        if (B->uploaded && cudaEventSynchronize(B->upload_done) != cudaSuccess) return AGJ_ECUDA;
        memcpy(B->h_jobs, jobs.data(), jobs.size() * sizeof(JobDesc));
        if (cudaMemcpyAsync(B->d_mem + S.off_jobs, B->h_jobs, jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            cudaEventRecord(B->upload_done, s) != cudaSuccess)
            return AGJ_ECUDA;
        B->last = jobs;
        B->uploaded = true;
    }
    const cudaError_t e = B->exec ? cudaGraphLaunch(B->exec, s) : enqueue(S, B->d_mem, B->ctas_per_sm, s);
    return e == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

// ---------------------------------------------------------------------------
// one launch for jobs formed on the fly (the served form)
// ---------------------------------------------------------------------------

int step_bytes(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, uint64_t* device_bytes,
               uint64_t* table_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    int rc = check_options(&ppt, 0);
    if (rc != AGJ_OK) return rc;
    Shape S;
    rc = make_shape(X, n, m, ppt, dev, &S);
    if (rc != AGJ_OK) return rc;
    *device_bytes = S.bytes;
    *table_bytes = S.table_bytes;
    return AGJ_OK;
}

int step_bound(uint64_t max_points, uint32_t max_jobs, int ppt, uint32_t max_cand_refs, uint64_t max_polys,
               bool exact, uint64_t* device_bytes, uint64_t* table_bytes) {
    int rc = check_options(&ppt, 0);
    if (rc != AGJ_OK) return rc;
    if (max_jobs > kMaxBatchJobs) return AGJ_EUNSUPPORTED;
    // every job adds at most one partial tile and the padding to a whole CTA
    const uint64_t T = (max_points + 32 * ppt - 1) / (32 * ppt) + (uint64_t)max_jobs * kWarpsPerBlock;
    const uint32_t slots = 32u * (uint32_t)ppt * std::max<uint32_t>(max_cand_refs, 1);
    if (max_polys >= 0xFFFFFFFFull || T * 32 * ppt >= 0xFFFFFFFFull || (exact && T * slots >= 0xFFFFFFFFull))
        return AGJ_ECAPACITY;
    const JoinLayout L = join_layout(T * 32 * ppt, T, exact, exact ? slots : 0u, exact ? max_polys : 0);
    const uint64_t m = std::max<uint32_t>(max_jobs, 1);
    *table_bytes = align256(m * sizeof(JobDesc)) + align256(T * 2 + 2);
    *device_bytes = *table_bytes + align256(m * 4) + align256(m * 16) + L.total;
    return AGJ_OK;
}

int step_enqueue(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int ctas_per_sm,
                 const double* const* d_points, agj_pairs* outs, void* d_work, uint64_t work_bytes, void* h_stage,
                 uint64_t stage_bytes, cudaStream_t s) {
    if (m == 0) return AGJ_OK;
    if (!X || !n || !d_points || !outs || !d_work || !h_stage) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_work) & 255u) != 0) return AGJ_EINVAL;
    int rc = check_options(&ppt, ctas_per_sm);
    if (rc != AGJ_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    Shape S;
    rc = make_shape(X, n, m, ppt, dev, &S);
    if (rc != AGJ_OK) return rc;
    if (S.bytes > work_bytes || S.table_bytes > stage_bytes) return AGJ_ECAPACITY;
    char* base = static_cast<char*>(d_work);
    char* stage = static_cast<char*>(h_stage);
    rc = fill_jobs(S, X, n, d_points, outs, reinterpret_cast<uint64_t*>(base + S.off_counters),
                   reinterpret_cast<JobDesc*>(stage + S.off_jobs));
    if (rc != AGJ_OK) return rc;
    fill_tile_job(S, reinterpret_cast<uint16_t*>(stage + S.off_tile_job));
    if (cudaMemcpyAsync(base, stage, S.table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return AGJ_ECUDA;
    return enqueue(S, base, ctas_per_sm, s) == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

}  // namespace agj
