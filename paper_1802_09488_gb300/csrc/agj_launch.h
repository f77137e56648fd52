// agj_launch.h — host entry points of the CUDA translation unit(s).
#pragma once

#include <cuda_runtime.h>

#include "agj_index.h"

namespace agj {

// Copies the flattened index and the polygons to one device allocation.
int upload_index(Index* X, cudaStream_t s);
// Size of that allocation (what upload_index would take).
uint64_t index_device_bytes(const Index& X);
int join_requirements(const Index& X, uint64_t n, agj_requirements* r);
// events: null, or 4 events recorded at the stage boundaries (see agj_join_timed).
int launch_join(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, agj_pairs* out,
                cudaEvent_t const* events = nullptr);
// Approximate join whose work space is a file-scope device array (no
// allocation); at most 2^24 points per call.
int launch_join_approx_noalloc(const Index& X, const double* d_points, uint64_t n, uint32_t* d_offsets,
                               uint32_t* d_ids, uint64_t ids_capacity, uint64_t* d_status, cudaStream_t s);
int launch_cell_ids(const double* d_points, uint64_t n, uint64_t* d_ids, cudaStream_t s);
// Aggregation mode (counts per polygon): work space size and the launch.
uint64_t count_scratch_bytes(const Index& X, uint64_t n);
int launch_join_count(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, uint64_t* d_counts,
                      uint64_t* d_status, void* scratch, uint64_t scratch_bytes, bool accumulate,
                      cudaEvent_t const* events = nullptr);
// Online training's device pass: the FP64 leaf ids of the points (n, device)
// whose cell holds a candidate reference go to d_out[0 .. *d_count) (d_out
// holds n ids; *d_count must start at 0; d_status: 4 zeroed words whose [1]
// collects device-side error bits).
int launch_collect_expensive(const Index& X, const double* d_points, uint64_t n, uint64_t* d_out,
                             uint64_t* d_count, uint64_t* d_status, cudaStream_t s);
// FP64 fused multiply-add throughput of the current device (flop/s), from
// an own kernel of independent FMA chains timed with events (synchronises).
int measure_fp64_rate(cudaStream_t s, double* flops_per_s);
// Runs the tile scan with a predecessor that never publishes (see agj.h).
int selftest_scan_timeout(cudaStream_t s);
int selftest_ready_timeout(cudaStream_t s);

// Batched form (agj_batch.cu): a plan for m (index, point count) jobs with
// its own work space and, with use_graph, an instantiated CUDA graph.
struct Batch;
int batch_create(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int ctas_per_sm, bool use_graph,
                 Batch** out);
int batch_run(Batch* B, const double* const* d_points, cudaStream_t s, agj_pairs* outs);
uint64_t batch_device_bytes(const Batch* B);
void batch_free(Batch* B);
// One batched launch for jobs formed on the fly (the served form): device
// work space (256-byte aligned) and pinned staging sizes for the jobs, and
// the launch itself on stream s (the staging buffer must stay untouched
// until the stream passes the launch).
int step_bytes(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, uint64_t* device_bytes,
               uint64_t* table_bytes);
// Work space and staging that suffice for any step of at most max_points
// points in max_jobs jobs over indexes with at most max_cand_refs candidate
// references per cell and max_polys polygons over the exact indexes.
int step_bound(uint64_t max_points, uint32_t max_jobs, int ppt, uint32_t max_cand_refs, uint64_t max_polys,
               bool exact, uint64_t* device_bytes, uint64_t* table_bytes);
int step_enqueue(const Index* const* X, const uint64_t* n, uint32_t m, int ppt, int ctas_per_sm,
                 const double* const* d_points, agj_pairs* outs, void* d_work, uint64_t work_bytes, void* h_stage,
                 uint64_t stage_bytes, cudaStream_t s);

}  // namespace agj
