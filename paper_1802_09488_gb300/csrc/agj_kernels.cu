// agj_kernels.cu — the plain join's launchers (§III-E), the kernels that are
// not templates (zeroing, scans, scatter, cell ids), the index upload and the
// allocation-free approximate join.  The probe, refine and emit kernels are
// in agj_probe.cuh; the plain join runs them on one job:
//
//   k_probe<approx>  per warp tile (128 points from 2^21 points on, 64 below):
//                    point loads, cell id, face/prefix stage, trie walk
//                    (Listing "Probe Adaptive Cell Trie"); stores each
//                    point's tagged entry and the tile's reference count
//   k_scan_counts    exclusive scan of tile counts (decoupled look-back over
//                    CTA chunks of 4096 tiles)
//   k_emit<approx>   offsets and ids (every reference: §V "approx")
//   k_probe<exact>   the same walk; true hits counted, candidate references
//                    compacted by warp ballot into a queue
//   k_count          candidates per polygon (shared histograms per chunk)
//   k_poly_scan      per-polygon candidate counts -> queue segments + chunks
//   k_scatter        queue grouped by polygon
//   k_pip            exact ST_Covers refine (§II "PIP"): one CTA per chunk of
//                    one polygon's candidates, the polygon's edges staged in
//                    shared memory and read by all threads (broadcast); adds
//                    passing candidates to their tile's pair count
//   k_scan_counts, k_emit<exact>   offsets and ids of the exact join
//   k_join_approx    probe, scan and emit in one pass with a per-tile
//                    look-back (the allocation-free entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "agj_index.h"
#include "agj_launch.h"
#include "agj_join.cuh"
#include "agj_probe.cuh"

namespace agj {

// ---------------------------------------------------------------------------
// kernels shared by the plain join and the batched form
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_zero(uint64_t* __restrict__ a, uint64_t na, uint64_t* __restrict__ b,
                                              uint64_t nb) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
        if (i < na) a[i] = 0;
        else b[i - na] = 0;
    }
}

// ORs the scan error bits into a status word (aggregation mode has no emit
// kernel to carry them).
__global__ void k_merge_err(const uint64_t* __restrict__ err, uint64_t* __restrict__ status_err) {
    if (threadIdx.x == 0 && *err) atomicOr((unsigned long long*)status_err, (unsigned long long)*err);
}

__global__ void k_cell_ids(const double2* __restrict__ pts, uint64_t n, uint64_t* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 p = pts[i];
        out[i] = point_cell_id(p.x, p.y);
    }
}

__global__ void __launch_bounds__(256) k_scan_counts(const uint32_t* __restrict__ tile_count, uint64_t m,
                                                     uint32_t* __restrict__ tile_prefix, uint64_t* __restrict__ chunks,
                                                     uint32_t* __restrict__ chunk_counter,
                                                     uint64_t* __restrict__ err,
                                                     const uint16_t* __restrict__ tile_job,
                                                     uint32_t* __restrict__ job_base) {
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_chunk;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_chunk = atomicAdd(chunk_counter, 1u);
    __syncthreads();
    const uint32_t chunk = s_chunk;
    const uint64_t i0 = (uint64_t)chunk * (256 * kScanItems) + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = i0 + k < m ? tile_count[i0 + k] : 0u;
        sum += v[k];
    }
    uint32_t total;
    const uint32_t excl = block_excl_scan<256>(sum, &total, s_warp);
    if (threadIdx.x < 32) {
        const uint64_t pre = lookback(chunks, chunk, total, err);
        if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint64_t o = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (i0 + k < m) {
            tile_prefix[i0 + k] = (uint32_t)o;
            if (tile_job) {
                const uint32_t j = tile_job[i0 + k];
                if (i0 + k == 0 || tile_job[i0 + k - 1] != j) job_base[j] = (uint32_t)o;
            }
        }
        o += v[k];
    }
}

constexpr int kPolyScanItems = 4;
__global__ void __launch_bounds__(256) k_poly_scan(const uint32_t* __restrict__ poly_count, uint32_t n_polys,
                                                   uint32_t* __restrict__ cursor, uint32_t* __restrict__ n_chunks,
                                                   uint4* __restrict__ chunk_desc, uint64_t* __restrict__ chunks,
                                                   uint32_t* __restrict__ chunk_counter, uint64_t* __restrict__ err) {
    __shared__ uint64_t s_warp[8];
    __shared__ uint32_t s_chunk;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_chunk = atomicAdd(chunk_counter, 1u);
    __syncthreads();
    const uint32_t chunk = s_chunk;
    const uint64_t i0 = (uint64_t)chunk * (256 * kPolyScanItems) + (uint64_t)threadIdx.x * kPolyScanItems;
    uint64_t v[kPolyScanItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kPolyScanItems; ++k) {
        const uint32_t c = i0 + k < n_polys ? poly_count[i0 + k] : 0u;
        v[k] = (uint64_t)c | ((uint64_t)((c + kPipBlock - 1) / kPipBlock) << 32);
        sum += v[k];
    }
    uint64_t total;
    const uint64_t excl = block_excl_scan<256>(sum, &total, s_warp);
    if (threadIdx.x < 32) {
        const uint64_t pre = lookback(chunks, chunk, total, err);
        if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint64_t o = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kPolyScanItems; ++k) {
        if (i0 + k < n_polys) {
            cursor[i0 + k] = (uint32_t)o;
            // refine chunks of this polygon: (polygon, first candidate, candidates)
            const uint32_t c0 = (uint32_t)(o >> 32), nch = (uint32_t)(v[k] >> 32);
            const uint32_t q = (uint32_t)o, cnt = (uint32_t)v[k];
            for (uint32_t t = 0; t < nch; ++t)
                chunk_desc[c0 + t] = make_uint4((uint32_t)(i0 + k), q + t * kPipBlock,
                                                min((uint32_t)kPipBlock, cnt - t * kPipBlock), 0u);
        }
        o += v[k];
    }
    if (chunk == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t t = s_prefix + total;
        *n_chunks = (uint32_t)(t >> 32);
    }
}

// The candidates queued by a chunk of ct <= kChunkTiles tiles (tile t holds
// tile_cand[t] items from slot t x tile_slots) are numbered densely: the
// chunk's counts are scanned into s_off, and item i lives in the last tile
// whose offset is <= i.  Returns the chunk's item count (after a barrier).
constexpr int kChunkTiles = 512;
__device__ __forceinline__ uint32_t chunk_number(const uint32_t* __restrict__ tile_cand, uint64_t n_tiles,
                                                 uint32_t tile_slots, uint32_t ct, uint64_t c0, uint32_t* s_off,
                                                 uint32_t* s_warp) {
    constexpr int kPer = kChunkTiles / 256;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const uint32_t r = threadIdx.x * kPer + k;
        const uint64_t t = c0 + r;
        v[k] = r < ct && t < n_tiles ? min(tile_cand[t], tile_slots) : 0u;
        sum += v[k];
    }
    uint32_t total;
    uint32_t o = block_excl_scan<256>(sum, &total, s_warp);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        s_off[threadIdx.x * kPer + k] = o;
        o += v[k];
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ uint64_t chunk_slot(const uint32_t* s_off, uint64_t c0, uint32_t tile_slots, uint32_t ct,
                                               uint32_t i) {
    uint32_t lo = 0, hi = ct;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off[mid] <= i) lo = mid; else hi = mid;
    }
    return (c0 + lo) * tile_slots + (i - s_off[lo]);
}

// Candidates per polygon: a shared-memory histogram per chunk, added to the
// global counts with one atomic per polygon and chunk (global atomics per
// item beyond kCountMaxPolys polygons, where they rarely collide).
constexpr int kCountMaxPolys = 8192;
__global__ void __launch_bounds__(256) k_count(const uint2* __restrict__ queue, const uint32_t* __restrict__ tile_cand,
                                               uint64_t n_tiles, uint32_t tile_slots, uint32_t ct,
                                               uint32_t* __restrict__ poly_count, uint32_t n_polys) {
    __shared__ uint32_t s_cnt[kCountMaxPolys];
    __shared__ uint32_t s_off[kChunkTiles];
    __shared__ uint32_t s_warp[8];
    const bool shared_counts = n_polys <= (uint32_t)kCountMaxPolys;
    if (shared_counts)
        for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x) s_cnt[p] = 0;
    for (uint64_t c0 = (uint64_t)blockIdx.x * ct; c0 < n_tiles; c0 += (uint64_t)gridDim.x * ct) {
        const uint32_t total = chunk_number(tile_cand, n_tiles, tile_slots, ct, c0, s_off, s_warp);
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
            const uint32_t poly = queue[chunk_slot(s_off, c0, tile_slots, ct, i)].y;
            if (shared_counts) atomicAdd(&s_cnt[poly], 1u);
            else atomicAdd(&poly_count[poly], 1u);
        }
        __syncthreads();
    }
    if (shared_counts) {
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x)
            if (s_cnt[p]) atomicAdd(&poly_count[p], s_cnt[p]);
    }
}

// Groups the queued candidates by polygon (counting-sort scatter of queue
// slots): per chunk, the items are counted per polygon in shared memory,
// each polygon's slots are reserved with one global atomic, and the items
// are written there.  With more polygons than shared counters, every item
// reserves its slot globally.
constexpr int kScatterMaxPolys = 4096;
__global__ void __launch_bounds__(256) k_scatter(const uint2* __restrict__ queue, const uint32_t* __restrict__ tile_cand,
                                                 uint64_t n_tiles, uint32_t tile_slots, uint32_t ct,
                                                 uint32_t* __restrict__ cursor, uint2* __restrict__ sorted,
                                                 uint32_t n_polys) {
    __shared__ uint32_t s_cnt[kScatterMaxPolys];
    __shared__ uint32_t s_base[kScatterMaxPolys];
    __shared__ uint32_t s_off[kChunkTiles];
    __shared__ uint32_t s_warp[8];
    const bool shared_counts = n_polys <= (uint32_t)kScatterMaxPolys;
    for (uint64_t c0 = (uint64_t)blockIdx.x * ct; c0 < n_tiles; c0 += (uint64_t)gridDim.x * ct) {
        if (shared_counts)
            for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x) s_cnt[p] = 0;
        const uint32_t total = chunk_number(tile_cand, n_tiles, tile_slots, ct, c0, s_off, s_warp);
        if (shared_counts) {
            for (uint32_t i = threadIdx.x; i < total; i += blockDim.x)
                atomicAdd(&s_cnt[queue[chunk_slot(s_off, c0, tile_slots, ct, i)].y], 1u);
            __syncthreads();
            for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x) {
                const uint32_t c = s_cnt[p];
                if (c) s_base[p] = atomicAdd(&cursor[p], c);
                s_cnt[p] = 0;
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
                const uint64_t q = chunk_slot(s_off, c0, tile_slots, ct, i);
                const uint2 it = queue[q];
                sorted[s_base[it.y] + atomicAdd(&s_cnt[it.y], 1u)] = make_uint2(it.x, (uint32_t)q);
            }
        } else {
            for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
                const uint64_t q = chunk_slot(s_off, c0, tile_slots, ct, i);
                const uint2 it = queue[q];
                sorted[atomicAdd(&cursor[it.y], 1u)] = make_uint2(it.x, (uint32_t)q);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// aggregation mode: count(*) group by polygon
// ---------------------------------------------------------------------------
// The paper's benchmark query (§V) counts the points of each polygon; its
// SIMD aggregation (§IV) adds the references of a vector of points with
// gather/scatter and defers the rare lanes (several references, candidates)
// to a buffer.  Here a warp adds the references of its 32 lanes with one
// atomic per distinct polygon (lanes naming the same polygon are combined by
// __match_any_sync), into a shared-memory histogram per CTA that is added to
// the global counts once, when the persistent CTA is done; lookup-table
// cells (more than two references) are added lane by lane.  In exact mode
// only true hits are counted here; candidates go to the tile's queue region
// and are refined and counted by k_pip<..., true>.
constexpr uint32_t kAggSmemPolys = 4096;       // polygons counted in shared memory (16 KB)
constexpr uint32_t kNoPoly = 0xFFFFFFFFu;

// With the global counts (many polygons), one atomic per distinct polygon
// among the warp's lanes (kNoPoly: none); with the shared histogram, one
// shared atomic per lane (lanes on the same polygon are serialised by the
// shared-memory unit, which is cheaper than finding them).
__device__ __forceinline__ void agg_add_warp(uint32_t poly, uint32_t* s_hist, uint64_t* counts) {
    if (s_hist) {
        if (poly != kNoPoly) atomicAdd(&s_hist[poly], 1u);
        return;
    }
    const uint32_t active = __ballot_sync(kFull, poly != kNoPoly);
    if (poly == kNoPoly) return;
    const uint32_t peers = __match_any_sync(active, poly);
    if ((threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
        atomicAdd((unsigned long long*)&counts[poly], (unsigned long long)__popc(peers));
}

__device__ __forceinline__ void agg_add_lane(uint32_t poly, uint32_t* s_hist, uint64_t* counts) {
    if (s_hist) atomicAdd(&s_hist[poly], 1u);
    else atomicAdd((unsigned long long*)&counts[poly], 1ull);
}

// One warp tile (32 lanes x PPT points) of the aggregation: cell id, walk,
// then every counted reference added; *pairs, *gathers and *fallbacks
// accumulate the lane's totals across tiles.
template <int PPT, int MODE>
__device__ __forceinline__ void agg_tile(const JobDesc& J, const DevFace* faces, const uint16_t* s_hlut,
                                         const uint64_t* s_root, uint64_t wt, const JoinScratch& S, uint32_t* s_hist,
                                         uint64_t* counts, uint32_t* pairs, uint32_t* gathers, uint32_t* fallbacks,
                                         uint32_t* s_cand, uint4* tail, uint64_t* ready, const double2* loaded) {
    constexpr bool exact = MODE == kModeExact;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t base = wt * (32 * PPT);
    PointIJ pij[PPT];
    bool ok[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        ok[k] = false;
        if (p < J.n) {
            const double2 q = loaded ? loaded[k] : __ldcs(J.pts + p);      // streamed once
            ok[k] = point_ij(J.X.model, q.x, q.y, false, pij[k]);
        }
    }
    // the shared tables (see probe_tile: a wait that gives up leaves the
    // tile's points unjoined and reports it)
    if (ready && !ready_wait(ready)) {
        if (lane == 0) atomicOr((unsigned long long*)&J.status[1], (unsigned long long)kErrScanTimeout);
#pragma unroll
        for (int k = 0; k < PPT; ++k) ok[k] = false;
    }
    uint64_t e[PPT];
    *gathers += probe_cells<PPT>(J.X, faces, s_hlut, s_root, pij, ok, J.pts + base + lane, e, &J.status[1], fallbacks,
                                 tail);
    uint32_t nc[PPT], csum = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt;
        entry_counts(J.X, e[k], &nt, &nc[k]);
        *pairs += exact ? nt : nt + nc[k];
        csum += exact ? nc[k] : 0u;
        const uint32_t tag = (uint32_t)(e[k] & 3ull);
        // one or two inline references (the second round only when a lane
        // of the warp holds two)
        {
            uint32_t poly = kNoPoly;
            if (tag == 1 || tag == 2) {
                const uint32_t pl = payload_of(e[k], 0);
                if (pl != kInvalidPayloadDev && (!exact || (pl & 1u))) poly = out_poly(J.X, pl >> 1);
            }
            agg_add_warp(poly, s_hist, counts);
        }
        if (__any_sync(kFull, tag == 2)) {
            uint32_t poly = kNoPoly;
            if (tag == 2) {
                const uint32_t pl = payload_of(e[k], 1);
                if (!exact || (pl & 1u)) poly = out_poly(J.X, pl >> 1);
            }
            agg_add_warp(poly, s_hist, counts);
        }
        // a lookup-table cell: its lists, lane by lane (rare)
        if (tag == 3) {
            const uint32_t off = payload_of(e[k], 0);
            const uint32_t nt3 = __ldg(J.X.lut + off);
            for (uint32_t t = 0; t < nt3; ++t) agg_add_lane(out_poly(J.X, __ldg(J.X.lut + off + 1 + t)), s_hist, counts);
            if (!exact) {
                const uint32_t nc3 = __ldg(J.X.lut + off + 1 + nt3);
                for (uint32_t t = 0; t < nc3; ++t)
                    agg_add_lane(out_poly(J.X, __ldg(J.X.lut + off + 2 + nt3 + t)), s_hist, counts);
            }
        }
    }
    if constexpr (exact) queue_tile<PPT>(J, e, nc, csum, wt, base, 0, S, s_cand);
}

// One warp per tile, eight tiles per CTA (the plain probe's grid).  With
// n_polys <= kAggSmemPolys the CTA counts into a shared histogram and, at
// its end, adds the non-zero counters to one of kAggStripes striped global
// copies (the CTA's block index picks it, spreading the atomics over the
// L2); k_agg_reduce sums the stripes.  With more polygons the warps add to
// the global counts directly.  Pair, trie-entry and fallback totals go
// through shared counters, one global atomic each per CTA.
template <int PPT, int MODE>
__global__ void __launch_bounds__(kJoinBlock, MODE == kModeApprox ? AGJ_APPROX_PROBE_MIN_BLOCKS : AGJ_PROBE_MIN_BLOCKS)
    k_agg_probe(const JobDesc J, uint64_t T, const JoinScratch S, uint64_t* __restrict__ counts,
                uint32_t* __restrict__ stripes) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint32_t s_hist[kAggSmemPolys];
    __shared__ uint32_t s_tot[4];           // pairs, trie entries read, FP64 fallbacks; [3] candidates (queue_tile [2])
    __shared__ uint4 s_tail[kWarpsPerBlock][32 * PPT];
    __shared__ uint64_t s_ready;
    const bool smem = stripes != nullptr;
    const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    // exact: as in the plain probe, the tile's point loads first, then the
    // histogram and counters zeroed and the tables-ready barrier set up
    // before the CTA's barrier.  Approximate: one CTA barrier after the
    // setup (the ready barrier measured 4 % slower there: 1.80 against
    // 1.73 ms per 1e8 city points).
    constexpr bool kReady = AGJ_PROBE_READY_BARRIER && MODE == kModeExact;
    double2 q[PPT];
    if (kReady) load_tile_points<PPT>(J, wt, wt < T, q);
    if (smem)
        for (uint32_t p = threadIdx.x; p < J.X.n_out_polys; p += blockDim.x) s_hist[p] = 0;
    uint64_t* ready = nullptr;
    if (kReady) ready = cta_begin(s_tot, 4, &s_ready);
    else if (threadIdx.x < 4) s_tot[threadIdx.x] = 0;
    const uint64_t* s_root = cta_setup_async(J.X, s_hlut, s_faces, s_rootbuf, ready);
    if (!ready) {
        cp_async_wait_all();
        __syncthreads();
    }
    if (wt < T) {
        uint32_t pairs = 0, gathers = 0, fallbacks = 0;
        agg_tile<PPT, MODE>(J, s_faces, s_hlut, s_root, wt, S, smem ? s_hist : nullptr, counts, &pairs, &gathers,
                            &fallbacks, s_tot + 1, s_tail[threadIdx.x >> 5], ready, ready ? q : nullptr);
        const uint32_t wp = __reduce_add_sync(kFull, pairs), wg = __reduce_add_sync(kFull, gathers),
                       wf = __reduce_add_sync(kFull, fallbacks);
        if ((threadIdx.x & 31) == 0) {
            if (wp) atomicAdd(&s_tot[0], wp);
            if (wg) atomicAdd(&s_tot[1], wg);
            if (wf) atomicAdd(&s_tot[2], wf);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // no copy of the CTA's outlives it
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_tot[0]) atomicAdd((unsigned long long*)&J.status[0], (unsigned long long)s_tot[0]);
        if (s_tot[1]) atomicAdd((unsigned long long*)&J.status[3], (unsigned long long)s_tot[1]);
        if (s_tot[2]) atomicAdd((unsigned long long*)&J.counters[0], (unsigned long long)s_tot[2]);
        if (s_tot[3]) atomicAdd((unsigned long long*)&J.status[2], (unsigned long long)s_tot[3]);
    }
    if (smem) {
        uint32_t* stripe = stripes + (uint64_t)(blockIdx.x % kAggStripes) * J.X.n_out_polys;
        for (uint32_t p = threadIdx.x; p < J.X.n_out_polys; p += blockDim.x)
            if (s_hist[p]) atomicAdd(&stripe[p], s_hist[p]);
    }
}

// counts[p] += the sum of the stripes' counters of polygon p.
__global__ void __launch_bounds__(256) k_agg_reduce(const uint32_t* __restrict__ stripes, uint32_t n_polys,
                                                    uint64_t* __restrict__ counts) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_polys) return;
    uint64_t s = 0;
    for (uint32_t k = 0; k < kAggStripes; ++k) s += stripes[(uint64_t)k * n_polys + p];
    if (s) counts[p] += s;
}

// ---------------------------------------------------------------------------
// online training: the device pass
// ---------------------------------------------------------------------------
// Training (§III-D) splits the cells that hold candidate references, in the
// order of how many training points hit them.  Only points inside such
// cells can hit one in any pass (splitting a cell partitions its points), so
// the device walks the whole stream and hands the host just those points'
// FP64 leaf ids (the spec the host trainer uses), compacted by warp ballot
// with one atomic per warp and point slot.
__global__ void __launch_bounds__(kJoinBlock, AGJ_PROBE_MIN_BLOCKS)
    k_collect_expensive(const JobDesc J, uint64_t T, uint64_t* __restrict__ out,
                        unsigned long long* __restrict__ count, uint64_t cap) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint4 s_tail[kWarpsPerBlock][32 * kJoinSmallPPT];
    const uint64_t* s_root = cta_setup_async(J.X, s_hlut, s_faces, s_rootbuf);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const bool active = wt < T;
    const uint64_t base = wt * (32 * kJoinSmallPPT);
    PointIJ pij[kJoinSmallPPT];
    bool ok[kJoinSmallPPT];
#pragma unroll
    for (int k = 0; k < kJoinSmallPPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        ok[k] = false;
        if (active && p < J.n) {
            const double2 q = __ldcs(J.pts + p);
            ok[k] = point_ij(J.X.model, q.x, q.y, false, pij[k]);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (!active) return;
    uint64_t e[kJoinSmallPPT];
    uint32_t fallbacks = 0;
    probe_cells<kJoinSmallPPT>(J.X, s_faces, s_hlut, s_root, pij, ok, J.pts + base + lane, e, &J.status[1], &fallbacks,
                          s_tail[threadIdx.x >> 5]);
#pragma unroll
    for (int k = 0; k < kJoinSmallPPT; ++k) {
        uint32_t nt, nc;
        entry_counts(J.X, e[k], &nt, &nc);
        const uint32_t mask = __ballot_sync(kFull, nc > 0);
        if (!mask) continue;
        unsigned long long o = 0;
        if (lane == 0) o = atomicAdd(count, (unsigned long long)__popc(mask));
        o = __shfl_sync(kFull, o, 0);
        if (nc > 0) {
            const uint64_t idx = o + __popc(mask & ((1u << lane) - 1u));
            const double2 q = J.pts[base + lane + 32 * k];
            if (idx < cap) out[idx] = point_cell_id(q.x, q.y);
        }
    }
}

// One-pass approximate join of the allocation-free entry point.  One warp
// tile = 32 lanes x PPT points.  Each warp scans its own tile and looks back
// on its own tile state, so no CTA barrier follows the setup.  Warp tiles are
// numbered from the CTA's ticket (the order CTAs started), which keeps the
// look-back free of deadlock.
constexpr int kNoAllocMinBlocks = 3;   // its PPT = 4 walks need the registers of 3 CTAs per SM
template <int PPT>
__global__ void __launch_bounds__(kJoinBlock, kNoAllocMinBlocks) k_join_approx(
    DevIndex X, const double2* __restrict__ pts, uint32_t n, uint32_t* __restrict__ offsets,
    uint32_t* __restrict__ ids, uint64_t ids_cap, uint64_t* __restrict__ tiles, uint32_t* __restrict__ tile_counter,
    uint64_t* __restrict__ status, uint64_t* __restrict__ fallback_counter) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint32_t s_cta;
    __shared__ uint4 s_tail[kWarpsPerBlock][32 * PPT];
    const uint64_t* s_root = cta_setup(&X, s_hlut, s_faces, s_rootbuf);
    if (threadIdx.x == 0) s_cta = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wt = s_cta * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint64_t base = (uint64_t)wt * (32 * PPT);
    if (base >= n) return;
    const uint32_t n_wt = (uint32_t)((n + 32 * PPT - 1) / (32 * PPT));
    double lat[PPT], lng[PPT];
    bool valid[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        valid[k] = p < n;
        const double2 q = valid[k] ? __ldcs(pts + p) : make_double2(0.0, 0.0);   // streamed once: evict first
        lat[k] = q.x;
        lng[k] = q.y;
    }
    uint64_t e[PPT];
    uint32_t fallbacks = 0;
    warp_count(probe_points<PPT>(X, s_faces, s_hlut, s_root, lat, lng, pts + base + lane, valid, e, &status[1],
                                 &fallbacks, s_tail[threadIdx.x >> 5]),
               &status[3]);
    warp_count(fallbacks, fallback_counter);
    uint32_t c[PPT], ex[PPT], run = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt, nc;
        entry_counts(X, e[k], &nt, &nc);
        c[k] = nt + nc;
        const uint32_t incl = warp_incl_scan(c[k]);
        ex[k] = run + incl - c[k];
        run += __shfl_sync(kFull, incl, 31);
    }
    const uint64_t prefix = lookback(tiles, wt, run, &status[1]);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!valid[k]) continue;
        const uint64_t p = base + lane + 32 * k;
        const uint64_t o = prefix + ex[k];
        __stcs(offsets + p, (uint32_t)o);
        if (c[k]) {
            if (o + c[k] <= ids_cap) emit_all(X, e[k], ids, o);
            else atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrIdsCapacity);
        }
    }
    if (wt == n_wt - 1 && lane == 0) {
        offsets[n] = (uint32_t)(prefix + run);
        status[0] = prefix + run;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Face table entry with the prefix decoded into its cell: the quadrant of
// each prefix level is the one whose Hilbert digit (under the orientation
// so far) matches the prefix's.
DevFace dev_face(int face, const FaceRoot& F) {
    DevFace d{F.root, F.prefix_bits, F.prefix, 0u, 0u, 0u, ((uint32_t)face & 1u) << 9};
    if (F.root == kNoRootDev) return d;
    const int L = (int)(F.prefix_bits / 2);
    uint32_t o = (uint32_t)face & 1u, pi = 0, pj = 0;
    for (int l = 0; l < L; ++l) {
        const uint32_t digit = (uint32_t)(F.prefix >> (2 * (L - 1 - l))) & 3u;
        for (uint32_t q = 0; q < 4; ++q) {
            uint32_t o2 = o;
            if (hilbert_digit(q >> 1, q & 1u, &o2) == digit) {
                pi = (pi << 1) | (q >> 1);
                pj = (pj << 1) | (q & 1u);
                o = o2;
                break;
            }
        }
    }
    const int sh = kLevels - L;
    d.pi = L ? pi << sh : 0u;
    d.pj = L ? pj << sh : 0u;
    d.pmask = L ? (0x3FFFFFFFu >> sh) << sh : 0u;
    d.o_row = o << 9;
    return d;
}

DevIndex make_dev_index(const Index& X) {
    DevIndex D;
    memset(&D, 0, sizeof D);
    const char* b = static_cast<const char*>(X.d_blob);
    D.nodes = reinterpret_cast<const uint64_t*>(b + X.off_nodes);
    D.lut = reinterpret_cast<const uint32_t*>(b + X.off_lut);
    D.poly_uv = reinterpret_cast<const double2*>(b + X.off_uv);
    D.poly_vkey = reinterpret_cast<const int64_t*>(b + X.off_vkey);
    D.poly_ukey = reinterpret_cast<const int64_t*>(b + X.off_ukey);
    D.poly_off = reinterpret_cast<const uint32_t*>(b + X.off_poff);
    D.poly_bbox = reinterpret_cast<const int64_t*>(b + X.off_bbox);
    D.poly_face = reinterpret_cast<const int8_t*>(b + X.off_face);
    D.poly_local = reinterpret_cast<const PolyLocal*>(b + X.off_plocal);
    D.poly_luv = reinterpret_cast<const F2*>(b + X.off_pluv);
    D.poly_band = reinterpret_cast<const uint16_t*>(b + X.off_pband);
    D.ring_off = reinterpret_cast<const uint32_t*>(b + X.off_roff);
    D.ring_end = reinterpret_cast<const uint32_t*>(b + X.off_rend);
    D.piece_poly = X.piece_poly.empty() ? nullptr : reinterpret_cast<const uint32_t*>(b + X.off_ppoly);
    D.n_nodes = X.nodes.size() / 256;
    D.n_lut = X.lut.size();
    D.n_polys = X.n_polys;
    D.n_out_polys = X.n_input_polys;
    D.max_depth = X.stats.max_depth;
    D.contains = X.contains ? 1u : 0u;
    for (int f = 0; f < 6; ++f) D.faces[f] = dev_face(f, X.faces[f]);
    D.model = X.model;
    return D;
}

namespace {

// Byte offsets of the sections of an index's device blob (256-byte aligned).
struct BlobLayout {
    uint64_t nodes, lut, uv, vkey, ukey, poff, bbox, face, plocal, pluv, pband, roff, rend, ppoly, total;
};

BlobLayout blob_layout(const Index& X) {
    const uint64_t nv = X.poly_off.empty() ? 0 : X.poly_off.back();
    BlobLayout B;
    uint64_t o = 0;
    B.nodes = o; o += align256(X.nodes.size() * 8 + 8);
    B.lut = o; o += align256(X.lut.size() * 4 + 4);
    B.uv = o; o += align256(nv * 16 + 16);
    B.vkey = o; o += align256(nv * 8 + 8);
    B.ukey = o; o += align256(nv * 8 + 8);
    B.poff = o; o += align256(X.poly_off.size() * 4 + 4);
    B.bbox = o; o += align256((uint64_t)X.n_polys * 32 + 32);
    B.face = o; o += align256((uint64_t)X.n_polys + 1);
    B.plocal = o; o += align256((uint64_t)X.n_polys * sizeof(PolyLocal) + 16);
    B.pluv = o; o += align256(nv * sizeof(F2) + 16);
    B.pband = o; o += align256(X.poly_band.size() * 2 + 16);
    B.roff = o; o += align256(X.ring_off.size() * 4 + 4);
    B.rend = o; o += align256(X.ring_end.size() * 4 + 4);
    B.ppoly = o; o += align256(X.piece_poly.size() * 4 + 4);
    B.total = o;
    return B;
}

}  // namespace

uint64_t index_device_bytes(const Index& X) { return blob_layout(X).total; }

int upload_index(Index* X, cudaStream_t s) {
    const uint64_t nv = X->poly_off.empty() ? 0 : X->poly_off.back();
    const BlobLayout B = blob_layout(*X);
    X->off_nodes = B.nodes; X->off_lut = B.lut; X->off_uv = B.uv; X->off_vkey = B.vkey; X->off_ukey = B.ukey;
    X->off_poff = B.poff; X->off_bbox = B.bbox; X->off_face = B.face; X->off_plocal = B.plocal;
    X->off_pluv = B.pluv; X->off_pband = B.pband; X->off_roff = B.roff; X->off_rend = B.rend;
    X->off_ppoly = B.ppoly;
    const uint64_t o = B.total;
    X->blob_bytes = o;
    std::vector<unsigned char> host(o, 0);
    auto put = [&](uint64_t off, const void* src, size_t bytes) {
        if (bytes) memcpy(host.data() + off, src, bytes);
    };
    put(X->off_nodes, X->nodes.data(), X->nodes.size() * 8);
    put(X->off_lut, X->lut.data(), X->lut.size() * 4);
    put(X->off_uv, X->poly_uv.data(), nv * 16);
    std::vector<int64_t> vk(nv), uk(nv), bb(4ull * X->n_polys);
    for (uint64_t t = 0; t < nv; ++t) {
        uk[t] = dkey(X->poly_uv[2 * t]);
        vk[t] = dkey(X->poly_uv[2 * t + 1]);
    }
    for (uint64_t t = 0; t < 4ull * X->n_polys; ++t) bb[t] = dkey(X->poly_bbox[t]);
    put(X->off_vkey, vk.data(), nv * 8);
    put(X->off_ukey, uk.data(), nv * 8);
    put(X->off_poff, X->poly_off.data(), X->poly_off.size() * 4);
    put(X->off_bbox, bb.data(), bb.size() * 8);
    put(X->off_face, X->poly_face.data(), X->poly_face.size());
    put(X->off_plocal, X->poly_local.data(), X->poly_local.size() * sizeof(PolyLocal));
    put(X->off_pluv, X->poly_luv.data(), X->poly_luv.size() * sizeof(F2));
    put(X->off_pband, X->poly_band.data(), X->poly_band.size() * 2);
    put(X->off_roff, X->ring_off.data(), X->ring_off.size() * 4);
    put(X->off_rend, X->ring_end.data(), X->ring_end.size() * 4);
    put(X->off_ppoly, X->piece_poly.data(), X->piece_poly.size() * 4);
    if (cudaMalloc(&X->d_blob, o) != cudaSuccess) { cudaGetLastError(); X->d_blob = nullptr; return AGJ_ENOMEM; }
    if (cudaMemcpyAsync(X->d_blob, host.data(), o, cudaMemcpyHostToDevice, s) != cudaSuccess) return AGJ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AGJ_ECUDA;
    X->stats.device_bytes = o;
    cudaGetDevice(&X->device);
    return AGJ_OK;
}

namespace {

int plain_ppt(uint64_t n) { return n >= kJoinWidePoints ? kJoinPPT : kJoinSmallPPT; }

JoinLayout plain_layout(const Index& X, uint64_t n, int ppt) {
    const uint64_t tiles = (n + 32 * ppt - 1) / (32 * ppt);
    const bool exact = X.mode == AGJ_EXACT;
    return join_layout(tiles * 32 * ppt, tiles, exact,
                       exact ? 32u * ppt * std::max<uint32_t>(X.stats.max_cand_refs, 1) : 0u,
                       exact ? X.n_polys : 0);
}

}  // namespace

// The work space stated for n points serves every join of at most n points:
// the larger of the layout n itself takes and the largest one a narrow
// (small-join) layout of fewer points takes.
int join_requirements(const Index& X, uint64_t n, agj_requirements* r) {
    r->ids_capacity = n * std::max<uint64_t>(X.stats.max_refs, 1);
    r->scratch_bytes = plain_layout(X, n, plain_ppt(n)).total;
    if (n >= kJoinWidePoints)
        r->scratch_bytes =
            std::max(r->scratch_bytes, plain_layout(X, kJoinWidePoints - 1, kJoinSmallPPT).total);
    return AGJ_OK;
}

JobDesc make_job(const Index& X, const double* d_points, uint64_t n, agj_pairs* out, uint64_t* counters) {
    JobDesc J;
    memset(&J, 0, sizeof J);
    J.X = make_dev_index(X);
    J.pts = reinterpret_cast<const double2*>(d_points);
    J.offsets = out->offsets;
    J.ids = out->ids;
    J.status = out->status;
    J.counters = counters;
    J.ids_cap = out->ids_capacity;
    J.n = (uint32_t)n;
    J.exact = X.mode == AGJ_EXACT ? 1u : 0u;
    return J;
}

int launch_cell_ids(const double* d_points, uint64_t n, uint64_t* d_ids, cudaStream_t s) {
    if (n == 0) return AGJ_OK;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sm_count() * 16);
    k_cell_ids<<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(d_points), n, d_ids);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

int launch_join(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, agj_pairs* out,
                cudaEvent_t const* events) {
    if (!out || !out->offsets || !out->status || (n && !d_points)) return AGJ_EINVAL;
    if (n >= 0xFFFFFFFFull) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return AGJ_EINVAL;
    const int ppt = plain_ppt(n);
    const JoinLayout L = plain_layout(X, n, ppt);
    agj_requirements req;
    join_requirements(X, n, &req);
    if (req.ids_capacity >= 0xFFFFFFFFull || L.queue_cap >= 0xFFFFFFFFull) return AGJ_ECAPACITY;   // 32-bit offsets
    if (!out->scratch || out->scratch_bytes < L.total || out->ids_capacity < req.ids_capacity ||
        (req.ids_capacity && !out->ids) || (reinterpret_cast<uintptr_t>(out->scratch) & 255u) != 0)
        return AGJ_ECAPACITY;
    char* sc = static_cast<char*>(out->scratch);
    OneJob src;
    src.d = make_job(X, d_points, n, out, reinterpret_cast<uint64_t*>(sc) + kHdrIdFallbacks);
    if (n == 0) {
        k_zero<<<1, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), L.zero_end / 8, out->status, 4);
        cudaMemsetAsync(out->offsets, 0, 4, s);
        if (events)
            for (int k = 0; k < 4; ++k) cudaEventRecord(events[k], s);
        return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    }
    JoinLaunch G;
    G.probe_grid = (int)((L.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);   // one warp per tile
    G.emit_grid = G.probe_grid;
    G.sms = sm_count();
    G.pip_grid = G.sms * AGJ_PIP_MIN_BLOCKS;
    const cudaError_t e =
        X.mode == AGJ_APPROX
            ? (ppt == kJoinPPT ? enqueue_join<kJoinPPT, OneJob, kModeApprox>(src, L, sc, G, out->status, 4, s, events)
                               : enqueue_join<kJoinSmallPPT, OneJob, kModeApprox>(src, L, sc, G, out->status, 4, s, events))
            : (ppt == kJoinPPT ? enqueue_join<kJoinPPT, OneJob, kModeExact>(src, L, sc, G, out->status, 4, s, events)
                               : enqueue_join<kJoinSmallPPT, OneJob, kModeExact>(src, L, sc, G, out->status, 4, s, events));
    return e == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

namespace {

JoinLayout count_layout(const Index& X, uint64_t n) {
    const uint64_t tiles = (n + 32 * kJoinSmallPPT - 1) / (32 * kJoinSmallPPT);
    const bool exact = X.mode == AGJ_EXACT;
    return join_layout(tiles * 32 * kJoinSmallPPT, tiles, exact,
                       exact ? 32u * kJoinSmallPPT * std::max<uint32_t>(X.stats.max_cand_refs, 1) : 0u,
                       exact ? X.n_polys : 0, true, X.n_input_polys <= kAggSmemPolys ? X.n_input_polys : 0);
}

}  // namespace

uint64_t count_scratch_bytes(const Index& X, uint64_t n) { return count_layout(X, n).total; }

int launch_join_count(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, uint64_t* d_counts,
                      uint64_t* d_status, void* scratch, uint64_t scratch_bytes, bool accumulate,
                      cudaEvent_t const* events) {
    if (!d_status || (X.n_input_polys && !d_counts) || (n && !d_points) || !scratch) return AGJ_EINVAL;
    if (n >= 0xFFFFFFFFull) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0 || (reinterpret_cast<uintptr_t>(scratch) & 255u) != 0)
        return AGJ_EINVAL;
    const JoinLayout L = count_layout(X, n);
    if (L.queue_cap >= 0xFFFFFFFFull) return AGJ_ECAPACITY;
    if (scratch_bytes < L.total) return AGJ_ECAPACITY;
    char* sc = static_cast<char*>(scratch);
    const JoinScratch S = join_scratch(L, sc);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sc);
    const int sms = sm_count();
    auto mark = [&](int k) {
        if (events) cudaEventRecord(events[k], s);
    };
    // zero the header, scan states and per-polygon candidate counts, the
    // status words and (unless accumulating) the counts
    {
        const uint64_t zw = L.zero_end / 8, cw = accumulate ? 0 : X.n_input_polys;
        const int grid = (int)std::min<uint64_t>((zw + cw + 4 + 255) / 256 + 1, (uint64_t)sms * 4);
        k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), zw, d_status, 4);
        if (cw) k_zero<<<grid, 256, 0, s>>>(d_counts, cw, nullptr, 0);
    }
    mark(0);
    agj_pairs none;
    memset(&none, 0, sizeof none);
    none.status = d_status;
    const JobDesc J = make_job(X, d_points, n, &none, reinterpret_cast<uint64_t*>(sc) + kHdrIdFallbacks);
    const bool exact = X.mode == AGJ_EXACT;
    uint32_t* stripes = L.stripes ? reinterpret_cast<uint32_t*>(sc + L.stripes) : nullptr;
    if (L.n_tiles) {
        const int grid = (int)((L.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
        if (exact) k_agg_probe<kJoinSmallPPT, kModeExact><<<grid, kJoinBlock, 0, s>>>(J, L.n_tiles, S, d_counts, stripes);
        else k_agg_probe<kJoinSmallPPT, kModeApprox><<<grid, kJoinBlock, 0, s>>>(J, L.n_tiles, S, d_counts, stripes);
        if (stripes)
            k_agg_reduce<<<(X.n_input_polys + 255) / 256, 256, 0, s>>>(stripes, X.n_input_polys, d_counts);
    }
    mark(1);
    if (exact && L.n_tiles && L.n_polys) {
        OneJob src;
        src.d = J;
        const uint32_t ct = refine_chunk_tiles(L.n_tiles, sms, L.n_polys);
        k_count<<<refine_sort_grid(L.n_tiles, ct, sms, AGJ_COUNT_CTAS_PER_SM), 256, 0, s>>>(
            S.queue, S.tile_cand, L.n_tiles, L.tile_slots, ct, S.poly_count, (uint32_t)L.n_polys);
        k_poly_scan<<<(unsigned)L.n_pchunks, 256, 0, s>>>(
            S.poly_count, (uint32_t)L.n_polys, reinterpret_cast<uint32_t*>(sc + L.cursor), hdr + 2,
            reinterpret_cast<uint4*>(sc + L.cpoly), reinterpret_cast<uint64_t*>(sc + L.pchunks), hdr + 3,
            reinterpret_cast<uint64_t*>(sc) + kHdrScanErr);
        k_scatter<<<refine_sort_grid(L.n_tiles, ct, sms, AGJ_SCATTER_CTAS_PER_SM), 256, 0, s>>>(
            S.queue, S.tile_cand, L.n_tiles, L.tile_slots, ct, reinterpret_cast<uint32_t*>(sc + L.cursor),
            reinterpret_cast<uint2*>(sc + L.sorted), (uint32_t)L.n_polys);
        k_pip<OneJob, true><<<sms * AGJ_PIP_MIN_BLOCKS, kPipBlock, 0, s>>>(
            src, 32 * kJoinSmallPPT, reinterpret_cast<const uint2*>(sc + L.sorted), reinterpret_cast<const uint4*>(sc + L.cpoly),
            hdr + 2, nullptr, nullptr, d_counts);
        // the polygon scan's wait status goes to the join's error word
        k_merge_err<<<1, 32, 0, s>>>(reinterpret_cast<const uint64_t*>(sc) + kHdrScanErr, d_status + 1);
    }
    mark(2);
    mark(3);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

int launch_collect_expensive(const Index& X, const double* d_points, uint64_t n, uint64_t* d_out,
                             uint64_t* d_count, uint64_t* d_status, cudaStream_t s) {
    if (n == 0) return AGJ_OK;
    const uint64_t tiles = (n + 32 * kJoinSmallPPT - 1) / (32 * kJoinSmallPPT);
    agj_pairs none;
    memset(&none, 0, sizeof none);
    none.status = d_status;
    const JobDesc J = make_job(X, d_points, n, &none, d_status + 2);    // diagnostics land in status[2..3]
    k_collect_expensive<<<(unsigned)((tiles + kWarpsPerBlock - 1) / kWarpsPerBlock), kJoinBlock, 0, s>>>(
        J, tiles, d_out, reinterpret_cast<unsigned long long*>(d_count), n);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

// ---------------------------------------------------------------------------
// FP64 throughput (a measurement utility for the cell-id kernel's roofline)
// ---------------------------------------------------------------------------
// Each thread runs kFmaChains independent chains of x = x * a + b (one
// rounding each, __fma_rn), so the FP64 pipe has independent work every
// cycle; 2 flops per FMA.  The result is stored so nothing is removed.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) k_fp64_fma(double a, double b, uint32_t iters, double* __restrict__ out) {
    double x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (uint32_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;       // practically never true; keeps the chains live
}

int measure_fp64_rate(cudaStream_t s, double* flops_per_s) {
    if (!flops_per_s) return AGJ_EINVAL;
    double* d = nullptr;
    if (cudaMalloc(&d, 64) != cudaSuccess) { cudaGetLastError(); return AGJ_ENOMEM; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sm_count() * 8;
    const uint32_t iters = 1u << 14;
    k_fp64_fma<<<grid, 256, 0, s>>>(0.999999, 1e-7, 256, d);        // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, s);
        k_fp64_fma<<<grid, 256, 0, s>>>(0.999999, 1e-7, iters, d);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms < best ? ms : best;
    }
    const int rc = cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    *flops_per_s = 2.0 * kFmaChains * (double)iters * grid * 256.0 / (best * 1e-3);
    return rc;
}

// ---------------------------------------------------------------------------
// self-test of the bounded waits
// ---------------------------------------------------------------------------
// The tile scan's look-back waits for its predecessor chunks with a bounded
// spin.  Here one CTA runs the scan as chunk 1 (its ticket counter starts
// at 1) while chunk 0's state is never published: the wait must run out,
// set kErrScanTimeout and return, leaving the context usable.
int selftest_scan_timeout(cudaStream_t s) {
    constexpr uint64_t kTiles = 2 * 256 * kScanItems;     // two chunks' worth of tiles
    char* d = nullptr;
    const uint64_t bytes = 256 + 256 + kTiles * 8;
    if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return AGJ_ENOMEM; }
    uint32_t* counter = reinterpret_cast<uint32_t*>(d);
    uint64_t* err = reinterpret_cast<uint64_t*>(d) + 1;
    uint64_t* chunks = reinterpret_cast<uint64_t*>(d + 256);
    uint32_t* counts = reinterpret_cast<uint32_t*>(d + 512);
    uint32_t* prefix = counts + kTiles;
    const uint32_t one = 1;
    int rc = AGJ_OK;
    if (cudaMemsetAsync(d, 0, bytes, s) != cudaSuccess ||
        cudaMemcpyAsync(counter, &one, 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = AGJ_ECUDA;
    if (rc == AGJ_OK) {
        k_scan_counts<<<1, 256, 0, s>>>(counts, kTiles, prefix, chunks, counter, err, nullptr, nullptr);
        uint64_t e = 0;
        if (cudaMemcpyAsync(&e, err, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = AGJ_ECUDA;
        else
            rc = (e & kErrScanTimeout) ? AGJ_ETIMEOUT : AGJ_OK;
    }
    cudaStreamSynchronize(s);
    cudaFree(d);
    return rc;
}

// The probe's wait for its CTA's shared tables (ready_wait) is bounded the
// same way.  Here one CTA stages its tables as the probe does, on a
// tables-ready barrier that expects one arrival more than the staging
// makes, so the phase never completes: every warp's wait must run out and
// report kErrScanTimeout.  The index is all zero (no fast model), so the
// staging copies only the Hilbert table.
__global__ void __launch_bounds__(kJoinBlock) k_selftest_ready(const DevIndex X, uint64_t* __restrict__ err) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint64_t s_ready;
    if (threadIdx.x == 0) ready_init(&s_ready, kReadyArrivals + 1);
    __syncthreads();
    cta_setup_async(X, s_hlut, s_faces, s_rootbuf, &s_ready);
    const bool ok = ready_wait(&s_ready);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr((unsigned long long*)err, (unsigned long long)kErrScanTimeout);
    asm volatile("cp.async.wait_all;" ::: "memory");
}

int selftest_ready_timeout(cudaStream_t s) {
    uint64_t* d = nullptr;
    if (cudaMalloc(&d, 8) != cudaSuccess) { cudaGetLastError(); return AGJ_ENOMEM; }
    DevIndex X;
    memset(&X, 0, sizeof X);
    int rc = cudaMemsetAsync(d, 0, 8, s) == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    if (rc == AGJ_OK) {
        k_selftest_ready<<<1, kJoinBlock, 0, s>>>(X, d);
        uint64_t e = 0;
        if (cudaMemcpyAsync(&e, d, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            rc = AGJ_ECUDA;
        else
            rc = (e & kErrScanTimeout) ? AGJ_ETIMEOUT : AGJ_OK;
    }
    cudaStreamSynchronize(s);
    cudaFree(d);
    return rc;
}

// ---------------------------------------------------------------------------
// approximate join without any allocation
// ---------------------------------------------------------------------------
// The one-pass approximate join needs work space for its tile scan: a
// 256-byte header (the tile counter) and one 8-byte state per tile of
// kNoAllocTile points.  For callers that must not allocate, that work space is this
// file-scope device array, sized for joins of up to kNoAllocMaxPoints points
// (131072 warp tiles of 128 points: 1 MiB + 256 B).  Every device that loads the library holds
// one copy until the process exits.  All calls on a device share it, so
// calls whose kernels overlap on the GPU race; the header and the tile
// states a call uses are cleared at the start of every call.
constexpr uint64_t kNoAllocMaxPoints = 1ull << 24;
constexpr uint64_t kNoAllocHeaderWords = 32;
constexpr int kNoAllocPPT = 4;
constexpr uint64_t kNoAllocTile = 32 * kNoAllocPPT;
constexpr uint64_t kNoAllocTiles = kNoAllocMaxPoints / kNoAllocTile;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocHeaderWords + kNoAllocTiles];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  The host-side
// name of the array is only a stand-in, so the address is looked up once per
// device with that device current and cached.
int noalloc_scratch(uint64_t** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return AGJ_ECUDA; }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return AGJ_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return AGJ_ECUDA; }
        g_noalloc_ptr[dev] = static_cast<uint64_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AGJ_OK;
}

}  // namespace

int launch_join_approx_noalloc(const Index& X, const double* d_points, uint64_t n, uint32_t* d_offsets,
                               uint32_t* d_ids, uint64_t ids_capacity, uint64_t* d_status, cudaStream_t s) {
    if (X.mode != AGJ_APPROX || !X.d_blob) return AGJ_EINVAL;
    if (!d_offsets || !d_status || (n && !d_points)) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return AGJ_EINVAL;
    if (n > kNoAllocMaxPoints) return AGJ_ECAPACITY;
    const uint64_t need = n * std::max<uint64_t>(X.stats.max_refs, 1);
    if (need >= 0xFFFFFFFFull) return AGJ_ECAPACITY;       // offsets are 32-bit, as in agj_join
    if (ids_capacity < need) return AGJ_ECAPACITY;
    if (need && !d_ids) return AGJ_EINVAL;
    uint64_t* sc = nullptr;
    const int rc = noalloc_scratch(&sc);
    if (rc != AGJ_OK) return rc;
    const uint64_t n_tiles = (n + kNoAllocTile - 1) / kNoAllocTile;
    const uint64_t zero_words = kNoAllocHeaderWords + n_tiles;
    {
        const int grid = (int)std::min<uint64_t>((zero_words + 255) / 256 + 1, (uint64_t)sm_count() * 4);
        k_zero<<<grid, 256, 0, s>>>(sc, zero_words, d_status, 4);
    }
    if (n == 0) {
        cudaMemsetAsync(d_offsets, 0, 4, s);
        return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    }
    const DevIndex D = make_dev_index(X);
    k_join_approx<kNoAllocPPT><<<(unsigned)((n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock), kJoinBlock, 0, s>>>(
        D, reinterpret_cast<const double2*>(d_points), (uint32_t)n, d_offsets, d_ids, need,
        sc + kNoAllocHeaderWords, reinterpret_cast<uint32_t*>(sc), d_status, sc + 2);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

}  // namespace agj
