// agj_batch.cu — the batched form of the probe (no counterpart in the paper):
// many (index, point batch) jobs of uneven sizes joined by one launch
// sequence whose probe and emit kernels are persistent grids striding over
// the jobs' warp tiles laid end to end, and whose refine step covers the
// candidate polygons of every exact job at once.  The sequence is captured
// once into a CUDA graph; a run uploads the job descriptors (only when a
// pointer changed) and launches the graph.
//
// Each job computes what the plain join computes for it, bit for bit: the
// same probe per point, the same candidate set and refine test, the same
// CSR (offsets of a job are differences of prefixes of its own tiles).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <new>
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

struct Batch {
    uint32_t m = 0;
    int ppt = 2;
    int ctas_per_sm = 0;                // 0: one warp per tile, else persistent grids
    bool use_graph = true;
    int device = 0;
    std::vector<const Index*> X;
    std::vector<uint64_t> n;
    std::vector<uint64_t> tile0;
    std::vector<uint32_t> poly0;
    JoinLayout L;
    // device: [job descriptors][job of each tile u16][job bases u32]
    // [poly0 u32 m+1][per-job counters 2 x u64][join work space]
    char* d_mem = nullptr;
    uint64_t off_jobs = 0, off_tile_job = 0, off_job_base = 0, off_poly0 = 0, off_counters = 0, off_scratch = 0,
             bytes = 0;
    JobDesc* h_jobs = nullptr;          // pinned staging of the descriptors
    std::vector<JobDesc> last;          // descriptors of the last upload
    bool uploaded = false;
    cudaEvent_t upload_done = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

template <int PPT>
cudaError_t enqueue_batch(Batch* B, cudaStream_t s) {
    ManyJobs src;
    src.d = reinterpret_cast<const JobDesc*>(B->d_mem + B->off_jobs);
    src.tile_job = reinterpret_cast<const uint16_t*>(B->d_mem + B->off_tile_job);
    src.base = reinterpret_cast<const uint32_t*>(B->d_mem + B->off_job_base);
    src.poly0 = reinterpret_cast<const uint32_t*>(B->d_mem + B->off_poly0);
    src.m = B->m;
    k_jobs_init<<<(B->m + 255) / 256, 256, 0, s>>>(src.d, B->m);
    JoinLaunch G;
    G.sms = sm_count();
    const uint64_t need = (B->L.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (B->ctas_per_sm == 0) {            // one warp per tile
        G.probe_grid = (int)std::max<uint64_t>(1, need);
        G.emit_grid = G.probe_grid;
    } else {                              // persistent grids
        G.probe_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)G.sms * B->ctas_per_sm));
        // the emit is short and latency-bound: a full-occupancy grid
        G.emit_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)G.sms * 8));
    }
    G.pip_grid = G.sms * 4;
    G.tile_job = src.tile_job;
    G.job_base = reinterpret_cast<uint32_t*>(B->d_mem + B->off_job_base);
    return enqueue_join<PPT, ManyJobs, kModeAny>(src, B->L, B->d_mem + B->off_scratch, G, nullptr, 0, s, nullptr);
}

cudaError_t enqueue(Batch* B, cudaStream_t s) {
    switch (B->ppt) {
        case 1: return enqueue_batch<1>(B, s);
        case 4: return enqueue_batch<4>(B, s);
        default: return enqueue_batch<2>(B, s);
    }
}

}  // namespace

void batch_free(Batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    if (B->upload_done) cudaEventDestroy(B->upload_done);
    if (B->h_jobs) cudaFreeHost(B->h_jobs);
    if (B->d_mem) cudaFree(B->d_mem);
    delete B;
}

int batch_create(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int ctas_per_sm, bool use_graph,
                 Batch** out) {
    if (!out || (m && (!X || !n))) return AGJ_EINVAL;
    *out = nullptr;
    if (m > kMaxBatchJobs) return AGJ_EUNSUPPORTED;
    if (ppt == 0) ppt = 2;
    if (ppt != 1 && ppt != 2 && ppt != 4) return AGJ_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 8) return AGJ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    uint64_t T = 0, P = 0;
    uint32_t mcr = 1;    // most candidate references of a point over the exact jobs
    bool any_exact = false;
    Batch* B = new (std::nothrow) Batch();
    if (!B) return AGJ_ENOMEM;
    B->m = m;
    B->ppt = ppt;
    B->ctas_per_sm = ctas_per_sm;
    B->use_graph = use_graph;
    B->device = dev;
    B->X.assign(X, X + m);
    B->n.assign(n, n + m);
    for (uint32_t j = 0; j < m; ++j) {
        const Index* x = X[j];
        if (!x || !x->d_blob || x->device != dev || n[j] >= 0xFFFFFFFFull) { delete B; return AGJ_EINVAL; }
        const uint64_t ids = n[j] * std::max<uint64_t>(x->stats.max_refs, 1);
        if (ids >= 0xFFFFFFFFull) { delete B; return AGJ_ECAPACITY; }
        B->tile0.push_back(T);
        B->poly0.push_back((uint32_t)P);
        // whole CTAs per job: a CTA's tiles share one job
        T += (n[j] + 32 * ppt - 1) / (32 * ppt);
        T = (T + kWarpsPerBlock - 1) / kWarpsPerBlock * kWarpsPerBlock;
        if (x->mode == AGJ_EXACT) {
            any_exact = true;
            P += x->n_polys;
            mcr = std::max<uint32_t>(mcr, x->stats.max_cand_refs);
        }
    }
    const uint32_t slots = 32u * (uint32_t)ppt * mcr;
    if (P >= 0xFFFFFFFFull || (any_exact && T * slots >= 0xFFFFFFFFull) || T >= (1ull << 36)) {
        delete B;
        return AGJ_ECAPACITY;
    }
    B->tile0.push_back(T);
    B->poly0.push_back((uint32_t)P);
    B->L = join_layout(T * 32 * ppt, T, any_exact, any_exact ? slots : 0u, P);
    std::vector<uint16_t> tile_job(T);
    for (uint32_t j = 0; j < m; ++j)
        std::fill(tile_job.begin() + B->tile0[j], tile_job.begin() + B->tile0[j + 1], (uint16_t)j);
    uint64_t o = 0;
    B->off_jobs = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * sizeof(JobDesc));
    B->off_tile_job = o; o += align256(T * 2 + 2);
    B->off_job_base = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * 4);
    B->off_poly0 = o; o += align256((uint64_t)(m + 1) * 4);
    B->off_counters = o; o += align256((uint64_t)std::max<uint32_t>(m, 1) * 16);
    B->off_scratch = o; o += B->L.total;
    B->bytes = o;
    if (cudaMalloc(&B->d_mem, o) != cudaSuccess) { cudaGetLastError(); B->d_mem = nullptr; batch_free(B); return AGJ_ENOMEM; }
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
    // the job-space tables never change for a plan
    cudaError_t e = cudaSuccess;
    if (T)
        e = cudaMemcpyAsync(B->d_mem + B->off_tile_job, tile_job.data(), T * 2, cudaMemcpyHostToDevice, B->cap_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_mem + B->off_poly0, B->poly0.data(), (m + 1) * 4ull, cudaMemcpyHostToDevice,
                            B->cap_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->cap_stream);
    if (e != cudaSuccess) { cudaGetLastError(); batch_free(B); return AGJ_ECUDA; }
    if (use_graph && m) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e1 = enqueue(B, B->cap_stream);
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

uint64_t batch_device_bytes(const Batch* B) { return B ? B->bytes : 0; }

int batch_run(Batch* B, const double* const* d_points, cudaStream_t s, agj_pairs* outs) {
    if (!B) return AGJ_EINVAL;
    if (B->m == 0) return AGJ_OK;
    if (!d_points || !outs) return AGJ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != B->device) { cudaGetLastError(); return AGJ_EINVAL; }
    std::vector<JobDesc> jobs(B->m);
    uint64_t* counters = reinterpret_cast<uint64_t*>(B->d_mem + B->off_counters);
    for (uint32_t j = 0; j < B->m; ++j) {
        agj_pairs* o = &outs[j];
        const uint64_t n = B->n[j];
        const Index& x = *B->X[j];
        if (!o->offsets || !o->status || (n && !d_points[j])) return AGJ_EINVAL;
        if ((reinterpret_cast<uintptr_t>(d_points[j]) & 15u) != 0) return AGJ_EINVAL;
        const uint64_t need = n * std::max<uint64_t>(x.stats.max_refs, 1);
        if (o->ids_capacity < need || (need && !o->ids)) return AGJ_ECAPACITY;
        // diagnostics go where the plain join puts them when the caller
        // passes a work space, else to the plan's own words
        uint64_t* c = (o->scratch && o->scratch_bytes >= 32) ? static_cast<uint64_t*>(o->scratch) + 2 : counters + 2 * j;
        JobDesc J = make_job(x, d_points[j], n, o, c);
        J.tile0 = B->tile0[j];
        J.poly0 = B->poly0[j];
        jobs[j] = J;
    }
    const bool same = B->uploaded && memcmp(jobs.data(), B->last.data(), jobs.size() * sizeof(JobDesc)) == 0;
    if (!same) {
        // the staging buffer may still feed the previous upload
        if (B->uploaded && cudaEventSynchronize(B->upload_done) != cudaSuccess) return AGJ_ECUDA;
        memcpy(B->h_jobs, jobs.data(), jobs.size() * sizeof(JobDesc));
        if (cudaMemcpyAsync(B->d_mem + B->off_jobs, B->h_jobs, jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            cudaEventRecord(B->upload_done, s) != cudaSuccess)
            return AGJ_ECUDA;
        B->last = jobs;
        B->uploaded = true;
    }
    const cudaError_t e = B->exec ? cudaGraphLaunch(B->exec, s) : enqueue(B, s);
    return e == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

}  // namespace agj
