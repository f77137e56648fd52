// agj_kernels.cu — the plain join's launchers (§III-E), the kernels that are
// not templates (zeroing, scans, scatter, cell ids), the index upload and the
// allocation-free approximate join.  The probe, refine and emit kernels are
// in agj_probe.cuh; the plain join runs them on one job:
//
//   k_probe<approx>  per 64-point warp tile: cell id, face/prefix stage, trie
//                    walk (Listing "Probe Adaptive Cell Trie"); stores each
//                    point's tagged entry and the tile's reference count
//   k_scan_counts    exclusive scan of tile counts (decoupled look-back over
//                    CTA chunks of 4096 tiles)
//   k_emit<approx>   offsets and ids (every reference: §V "approx")
//   k_probe<exact>   the same walk; true hits counted, candidate references
//                    compacted by warp ballot into a queue
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
                                 &fallbacks),
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
    D.n_nodes = X.nodes.size() / 256;
    D.n_lut = X.lut.size();
    D.n_polys = X.n_polys;
    D.max_depth = X.stats.max_depth;
    for (int f = 0; f < 6; ++f) D.faces[f] = DevFace{X.faces[f].root, X.faces[f].prefix_bits, X.faces[f].prefix};
    D.model = X.model;
    return D;
}

int upload_index(Index* X, cudaStream_t s) {
    const uint64_t nv = X->poly_off.empty() ? 0 : X->poly_off.back();
    uint64_t o = 0;
    X->off_nodes = o; o += align256(X->nodes.size() * 8 + 8);
    X->off_lut = o; o += align256(X->lut.size() * 4 + 4);
    X->off_uv = o; o += align256(nv * 16 + 16);
    X->off_vkey = o; o += align256(nv * 8 + 8);
    X->off_ukey = o; o += align256(nv * 8 + 8);
    X->off_poff = o; o += align256(X->poly_off.size() * 4 + 4);
    X->off_bbox = o; o += align256((uint64_t)X->n_polys * 32 + 32);
    X->off_face = o; o += align256((uint64_t)X->n_polys + 1);
    X->off_plocal = o; o += align256((uint64_t)X->n_polys * sizeof(PolyLocal) + 16);
    X->off_pluv = o; o += align256(nv * sizeof(F2) + 16);
    X->off_pband = o; o += align256(X->poly_band.size() * 2 + 16);
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
    if (cudaMalloc(&X->d_blob, o) != cudaSuccess) { cudaGetLastError(); X->d_blob = nullptr; return AGJ_ENOMEM; }
    if (cudaMemcpyAsync(X->d_blob, host.data(), o, cudaMemcpyHostToDevice, s) != cudaSuccess) return AGJ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AGJ_ECUDA;
    X->stats.device_bytes = o;
    cudaGetDevice(&X->device);
    return AGJ_OK;
}

namespace {

JoinLayout plain_layout(const Index& X, uint64_t n) {
    const uint64_t tiles = (n + 32 * kJoinPPT - 1) / (32 * kJoinPPT);
    const bool exact = X.mode == AGJ_EXACT;
    return join_layout(tiles * 32 * kJoinPPT, tiles, exact,
                       exact ? 32u * kJoinPPT * std::max<uint32_t>(X.stats.max_cand_refs, 1) : 0u,
                       exact ? X.n_polys : 0);
}

}  // namespace

int join_requirements(const Index& X, uint64_t n, agj_requirements* r) {
    r->ids_capacity = n * std::max<uint64_t>(X.stats.max_refs, 1);
    r->scratch_bytes = plain_layout(X, n).total;
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
    const JoinLayout L = plain_layout(X, n);
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
            ? enqueue_join<kJoinPPT, OneJob, kModeApprox>(src, L, sc, G, out->status, 4, s, events)
            : enqueue_join<kJoinPPT, OneJob, kModeExact>(src, L, sc, G, out->status, 4, s, events);
    return e == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
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
