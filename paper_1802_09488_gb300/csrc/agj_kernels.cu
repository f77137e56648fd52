// agj_kernels.cu — sm_103a kernels of the probe side (§III-E) and their
// launchers.
//
//   k_cell_ids       point -> 64-bit cell id (FP64 spec of agj_geom.cuh)
//   k_probe_approx   per 128-point warp tile: cell id, face/prefix stage, trie
//                    walk (Listing "Probe Adaptive Cell Trie"); stores each
//                    point's tagged entry and the tile's reference count
//   k_scan_counts    exclusive scan of tile counts (decoupled look-back over
//                    CTA chunks of 4096 tiles)
//   k_emit_approx    offsets and ids (every reference: §V "approx")
//   k_join_approx    the same three steps in one pass with a per-tile
//                    look-back (used where no work space can be allocated)
//   k_probe_exact    cell id + walk + decode; true hits counted, candidate
//                    references compacted by warp ballot into a queue
//   k_poly_scan      per-polygon candidate counts -> queue segments + chunks
//   k_scatter        queue grouped by polygon
//   k_pip            exact ST_Covers refine (§II "PIP"): one CTA per chunk of
//                    one polygon's candidates, the polygon's edges staged in
//                    shared memory and read by all threads (broadcast); adds
//                    passing candidates to their tile's pair count
//   k_emit_exact     offsets and ids of the exact join
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "agj_device.cuh"
#include "agj_geom.cuh"
#include "agj_index.h"
#include "agj_launch.h"

namespace agj {

constexpr uint32_t kFull = 0xFFFFFFFFu;
__device__ const HilbertLut g_hilbert_lut = make_hilbert_lut();
constexpr uint32_t kSpinLimit = 1u << 22;
#ifndef AGJ_PROBE_MIN_BLOCKS
#define AGJ_PROBE_MIN_BLOCKS 3   // resident CTAs per SM the probe kernels are compiled for
#endif
constexpr int kJoinBlock = 256;
constexpr int kJoinPPT = 2;
constexpr int kWarpsPerBlock = kJoinBlock / 32;
constexpr int kTile = 32 * kJoinPPT;           // points per warp tile (scan granularity)
constexpr int kPipBlock = 256;
constexpr int kPipSmemVerts = 2048;           // vertices staged per pass (32 B each)

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------

template <int BLOCK>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = BLOCK / 32;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    *total = s_warp[NW - 1];
    const uint32_t wp = warp ? s_warp[warp - 1] : 0u;
    __syncthreads();
    return wp + x - v;
}

// Decoupled look-back across tiles (run by one full warp).  Tile states are
// 64-bit words: top 2 bits 0 = not ready, 1 = aggregate, 2 = inclusive
// prefix; low 62 bits the value.  Tiles are numbered in the order their CTAs
// started (atomic counter), so every predecessor is running or done and the
// wait ends; it is bounded all the same and reports kErrScanTimeout.
__device__ uint64_t lookback(uint64_t* tiles, uint32_t tile, uint64_t total, uint64_t* status) {
    const int lane = threadIdx.x & 31;
    constexpr uint64_t kVal = (1ull << 62) - 1ull;
    if (tile == 0) {
        if (lane == 0) st_release_u64(&tiles[0], (2ull << 62) | total);
        return 0;
    }
    if (lane == 0) st_release_u64(&tiles[tile], (1ull << 62) | total);
    uint64_t prefix = 0;
    int64_t idx = (int64_t)tile - 1;
    uint32_t spins = 0;
    for (;;) {
        const int64_t t = idx - lane;
        uint64_t st = 2ull << 62;
        if (t >= 0) {
            st = ld_acquire_u64(&tiles[t]);
            while ((st >> 62) == 0ull) {
                if (++spins > kSpinLimit) {
                    atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrScanTimeout);
                    st = 1ull << 62;
                    break;
                }
                __nanosleep(32);
                st = ld_acquire_u64(&tiles[t]);
            }
        }
        const uint32_t inc = __ballot_sync(kFull, (st >> 62) == 2ull);
        const int first = inc ? __ffs(inc) - 1 : 31;
        uint64_t c = lane <= first ? (st & kVal) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
        prefix += __shfl_sync(kFull, c, 0);
        if (inc) break;
        idx -= 32;
    }
    if (lane == 0) st_release_u64(&tiles[tile], (2ull << 62) | (prefix + total));
    return prefix;
}

// ---------------------------------------------------------------------------
// per-point probe: cell id -> face root -> common prefix -> trie walk
// ---------------------------------------------------------------------------

// Walk state of one point.  The key bytes of the leaf id are produced one at
// a time from the 4-level Hilbert table as the walk consumes them (byte b
// holds levels 4b+1 .. 4b+4).
struct Walk {
    uint32_t i32, j32;      // (i, j) << 2: levels 31-32 are zero padding
    uint32_t o;             // Hilbert orientation before byte b
    uint32_t b;             // next key byte
    uint32_t node;          // current trie node
    int32_t cert;           // key bytes whose levels are all certified
    int32_t st;             // 0 done, 1 walking, 2 needs the FP64 cell id
};

__device__ __forceinline__ uint32_t next_byte(const uint16_t* lut, Walk& w) {
    const uint32_t sh = 28u - 4u * w.b;
    const uint32_t e = lut[(w.o << 8) | (((w.i32 >> sh) & 15u) << 4) | ((w.j32 >> sh) & 15u)];
    w.o = e & 3u;
    ++w.b;
    return e >> 2;
}

// Cell id + face/prefix stage (§IV-B stage 1) for one point.  With the
// index's fast model (and exact == false) the id comes from the certified FP32
// path; otherwise from the FP64 spec.  Leaves w.st = 0 when the point joins
// nothing, 1 when the walk can start at w.node, 2 when an uncertified level
// decides the prefix.
__device__ __forceinline__ void begin_walk(const DevIndex& X, const DevFace* faces, const uint16_t* lut, double lat,
                                           double lng, bool exact, Walk& w) {
    uint32_t i, j;
    int lc, face;
    w.st = 0;
    w.b = 0;
    if (!exact && X.model.enabled) {
        if (!model_ij(X.model, lat, lng, &i, &j, &lc)) return;       // outside the window: in no cell
        face = X.model.face;
        if (lc >= kLevels) lc = kLevels + 2;                        // exact id: padding levels too
    } else {
        if (!point_valid(lat, lng)) return;
        double u, v;
        face = face_uv(lat, lng, &u, &v);
        i = st_to_ij(uv_to_st(u));
        j = st_to_ij(uv_to_st(v));
        lc = kLevels + 2;
    }
    const DevFace fr = faces[face];
    if (fr.root == kNoRootDev) return;
    w.i32 = i << 2;
    w.j32 = j << 2;
    w.o = (uint32_t)face & 1u;
    w.b = 0;
    w.cert = lc >> 2;
    const uint32_t nb = fr.prefix_bits >> 3;
    for (uint32_t q = 0; q < nb; ++q) {
        const uint32_t byte = next_byte(lut, w);
        if (byte != (uint32_t)((fr.prefix >> (8 * (nb - 1 - q))) & 0xFFu)) {
            w.st = (int32_t)q < w.cert ? 0 : 2;                     // certain mismatch: no cell
            return;
        }
    }
    if ((int32_t)nb > w.cert) { w.st = 2; return; }
    w.node = fr.root;
    w.st = 1;
}

// Walks of PPT points advance level by level together, so their gathers
// (Listing "Probe Adaptive Cell Trie") are in flight at the same time.
// Points whose walk needs an uncertified key byte get their FP64 id and walk
// again alone (counted in *fallbacks).  Returns the trie entries read.
template <int PPT>
__device__ __forceinline__ uint32_t probe_points(const DevIndex& X, const DevFace* faces, const uint16_t* lut,
                                                 const uint64_t* s_root, const double* lat, const double* lng,
                                                 const bool* valid, uint64_t e[PPT], uint64_t* err,
                                                 uint32_t* fallbacks) {
    uint32_t gathers = 0;
    Walk w[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        e[k] = 0;
        w[k].st = 0;
        w[k].b = 0;
        if (valid[k]) begin_walk(X, faces, lut, lat[k], lng[k], false, w[k]);
    }
    uint32_t prefix_bytes[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) prefix_bytes[k] = w[k].b;
    const uint32_t n_nodes32 = (uint32_t)min(X.n_nodes, (uint64_t)0xFFFFFFFFu);
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        uint64_t v[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            v[k] = 0;
            if (w[k].st == 1) {
                if (w[k].b >= (uint32_t)w[k].cert) {
                    w[k].st = 2;
                } else {
                    const uint32_t byte = next_byte(lut, w[k]);
                    // with the fast model every walk starts at the model face's root,
                    // which each CTA holds in shared memory
                    v[k] = (d == 0 && s_root) ? s_root[byte] : __ldg(X.nodes + (((uint64_t)w[k].node) << 8) + byte);
                }
            }
        }
        bool any = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (w[k].st != 1) continue;
            // child entries hold node << 11 with node < 2^32, so the low 32 bits
            // of (v >> 11) name the node; checking them keeps every read in bounds
            const uint32_t child = (uint32_t)(v[k] >> 11);
            if ((v[k] & 3ull) != 0ull || v[k] == 0ull) {
                e[k] = v[k];
                w[k].st = 0;
            } else if (child >= n_nodes32) {
                atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
                w[k].st = 0;
            } else {
                w[k].node = child;
                any = true;
            }
        }
        if (!any) break;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) gathers += w[k].b - prefix_bytes[k];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (w[k].st == 1) {
            atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
            e[k] = 0;
        } else if (w[k].st == 2) {
            ++*fallbacks;
            Walk x;
            begin_walk(X, faces, lut, lat[k], lng[k], true, x);
            e[k] = 0;
            while (x.st == 1) {
                if (x.b >= 8u) {
                    atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
                    break;
                }
                const uint32_t byte = next_byte(lut, x);
                const uint64_t v = __ldg(X.nodes + (((uint64_t)x.node) << 8) + byte);
                ++gathers;
                if ((v & 3ull) != 0ull || v == 0ull) {
                    e[k] = v;
                    break;
                }
                if ((v >> 11) >= X.n_nodes) {
                    atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
                    break;
                }
                x.node = (uint32_t)(v >> 11);
            }
        }
    }
    return gathers;
}

// Adds a per-thread count to a device counter with one atomic per warp.
__device__ __forceinline__ void warp_count(uint32_t v, uint64_t* counter) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)counter, (unsigned long long)v);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Per-CTA setup shared by the probe kernels: Hilbert table and face table in
// shared memory, and, with the fast model, the model face's root node.
// Returns the shared root (or null).
__device__ __forceinline__ const uint64_t* cta_setup(const DevIndex& X, uint16_t* s_hlut, DevFace* s_faces,
                                                     uint64_t* s_root) {
    for (int t = threadIdx.x; t < 512; t += blockDim.x)
        reinterpret_cast<uint32_t*>(s_hlut)[t] = reinterpret_cast<const uint32_t*>(g_hilbert_lut.v)[t];
    if (threadIdx.x < 6) s_faces[threadIdx.x] = X.faces[threadIdx.x];
    if (!s_root || !X.model.enabled) return nullptr;
    const uint32_t root = X.faces[X.model.face].root;
    if (root == kNoRootDev) return nullptr;
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(X.nodes + (uint64_t)root * 256);
    for (int t = threadIdx.x; t < 128; t += blockDim.x) reinterpret_cast<ulonglong2*>(s_root)[t] = __ldg(src + t);
    return s_root;
}

__device__ __forceinline__ uint32_t payload_of(uint64_t e, int which) {
    return (uint32_t)(e >> (which ? 33 : 2)) & 0x7FFFFFFFu;
}

// Writes every reference of entry e (approximate join), ascending ids.
__device__ __forceinline__ void emit_all(const DevIndex& X, uint64_t e, uint32_t* ids, uint64_t o) {
    const uint32_t tag = (uint32_t)(e & 3ull);
    if (tag == 1) {
        ids[o] = payload_of(e, 0) >> 1;
    } else if (tag == 2) {
        ids[o] = payload_of(e, 0) >> 1;
        ids[o + 1] = payload_of(e, 1) >> 1;
    } else if (tag == 3) {
        const uint32_t off = payload_of(e, 0);
        const uint32_t nt = __ldg(X.lut + off);
        const uint32_t* T = X.lut + off + 1;
        const uint32_t nc = __ldg(X.lut + off + 1 + nt);
        const uint32_t* Cc = X.lut + off + 2 + nt;
        uint32_t a = 0, b = 0;
        while (a < nt || b < nc) {
            const uint32_t ta = a < nt ? __ldg(T + a) : 0xFFFFFFFFu;
            const uint32_t cb = b < nc ? __ldg(Cc + b) : 0xFFFFFFFFu;
            if (ta < cb) { ids[o++] = ta; ++a; }
            else { ids[o++] = cb; ++b; }
        }
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void k_zero(uint64_t* __restrict__ a, uint64_t na, uint64_t* __restrict__ b, uint64_t nb) {
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

// One warp tile = 32 lanes x PPT points, point base + lane + 32 k, so the
// 16-byte point loads and the offset stores of a warp are contiguous.  Each
// warp scans its own tile and looks back on its own tile state, so no CTA
// barrier follows the setup.  Warp tiles are numbered from the CTA's ticket
// (the order CTAs started), which keeps the look-back free of deadlock.
template <int PPT>
__global__ void __launch_bounds__(kJoinBlock, AGJ_PROBE_MIN_BLOCKS) k_join_approx(DevIndex X, const double2* __restrict__ pts, uint32_t n,
                                                            uint32_t* __restrict__ offsets, uint32_t* __restrict__ ids,
                                                            uint64_t ids_cap, uint64_t* __restrict__ tiles,
                                                            uint32_t* __restrict__ tile_counter,
                                                            uint64_t* __restrict__ status,
                                                            uint64_t* __restrict__ fallback_counter) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint32_t s_cta;
    const uint64_t* s_root = cta_setup(X, s_hlut, s_faces, s_rootbuf);
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
    warp_count(probe_points<PPT>(X, s_faces, s_hlut, s_root, lat, lng, valid, e, &status[1], &fallbacks), &status[3]);
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
    const uint64_t prefix = lookback(tiles, wt, run, status);
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

// Exact-mode probe: entries + compacted candidate queue (warp ballot: one
// atomic reserves a warp's slots).
template <int PPT>
__global__ void __launch_bounds__(kJoinBlock, AGJ_PROBE_MIN_BLOCKS) k_probe_exact(DevIndex X, const double2* __restrict__ pts, uint32_t n,
                                                            uint64_t* __restrict__ entries, uint32_t* __restrict__ qbase,
                                                            uint2* __restrict__ queue, uint64_t queue_cap,
                                                            uint32_t* __restrict__ queue_len,
                                                            uint32_t* __restrict__ poly_count,
                                                            uint32_t* __restrict__ tile_count,
                                                            uint64_t* __restrict__ status,
                                                            uint64_t* __restrict__ fallback_counter) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    const uint64_t* s_root = cta_setup(X, s_hlut, s_faces, s_rootbuf);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t base = ((uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * (32 * PPT);
    if (base >= n) return;
    double lat[PPT], lng[PPT];
    bool valid[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        valid[k] = p < n;
        const double2 q = valid[k] ? __ldcs(pts + p) : make_double2(0.0, 0.0);
        lat[k] = q.x;
        lng[k] = q.y;
    }
    uint64_t e[PPT];
    uint32_t fallbacks = 0;
    warp_count(probe_points<PPT>(X, s_faces, s_hlut, s_root, lat, lng, valid, e, &status[1], &fallbacks), &status[3]);
    warp_count(fallbacks, fallback_counter);
    uint32_t nc[PPT], csum = 0, tsum = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt;
        entry_counts(X, e[k], &nt, &nc[k]);
        csum += nc[k];
        tsum += nt;
        if (valid[k]) entries[base + lane + 32 * k] = e[k];
    }
    // the tile's pair count starts at its true hits; the refine kernel adds the
    // candidates that pass
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(kFull, tsum, o);
    if (lane == 0) tile_count[base / (32 * PPT)] = tsum;
    const uint32_t x = warp_incl_scan(csum);
    const uint32_t wtotal = __shfl_sync(kFull, x, 31);
    if (wtotal == 0) return;
    uint32_t wbase = 0;
    if (lane == 0) {
        wbase = atomicAdd(queue_len, wtotal);
        atomicAdd((unsigned long long*)&status[2], (unsigned long long)wtotal);
    }
    wbase = __shfl_sync(kFull, wbase, 0);
    uint64_t q = (uint64_t)wbase + x - csum;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!nc[k]) continue;
        const uint32_t p = (uint32_t)(base + lane + 32 * k);
        qbase[p] = (uint32_t)q;
        const uint64_t ek = e[k];
        const uint32_t tag = (uint32_t)(ek & 3ull);
        if (tag == 1 || tag == 2) {
            for (int t = 0; t < (int)tag; ++t) {
                const uint32_t pl = payload_of(ek, t);
                if (pl & 1u) continue;
                if (q < queue_cap) { queue[q] = make_uint2(p, pl >> 1); atomicAdd(&poly_count[pl >> 1], 1u); }
                else atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrQueueOverflow);
                ++q;
            }
        } else {
            const uint32_t off = payload_of(ek, 0);
            const uint32_t nt = __ldg(X.lut + off);
            const uint32_t* Cc = X.lut + off + 2 + nt;
            for (uint32_t t = 0; t < nc[k]; ++t) {
                const uint32_t pg = __ldg(Cc + t);
                if (q < queue_cap) { queue[q] = make_uint2(p, pg); atomicAdd(&poly_count[pg], 1u); }
                else atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrQueueOverflow);
                ++q;
            }
        }
    }
}

// Approximate join, step 1: cell id + walk for every point of a warp tile;
// the tagged entry of each point is stored and the tile's number of
// references is counted (no waiting on other tiles).
template <int PPT>
__global__ void __launch_bounds__(kJoinBlock, AGJ_PROBE_MIN_BLOCKS) k_probe_approx(
    DevIndex X, const double2* __restrict__ pts, uint32_t n, uint64_t* __restrict__ entries,
    uint32_t* __restrict__ tile_count, uint64_t* __restrict__ status, uint64_t* __restrict__ fallback_counter) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    const uint64_t* s_root = cta_setup(X, s_hlut, s_faces, s_rootbuf);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint64_t base = wt * (32 * PPT);
    if (base >= n) return;
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
    warp_count(probe_points<PPT>(X, s_faces, s_hlut, s_root, lat, lng, valid, e, &status[1], &fallbacks), &status[3]);
    warp_count(fallbacks, fallback_counter);
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt, nc;
        entry_counts(X, e[k], &nt, &nc);
        c += nt + nc;
        if (valid[k]) entries[base + lane + 32 * k] = e[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    if (lane == 0) tile_count[wt] = c;
}

// Exclusive scan of the per-tile counts: CTA chunks of 16 x 256 counts, chained
// by the decoupled look-back (a few hundred chunks, so the look-back is short).
// The last chunk writes the total to offsets[n] and status[0].
constexpr int kScanItems = 16;
__global__ void __launch_bounds__(256) k_scan_counts(const uint32_t* __restrict__ tile_count, uint64_t m,
                                                     uint32_t* __restrict__ tile_prefix, uint64_t* __restrict__ chunks,
                                                     uint32_t* __restrict__ chunk_counter, uint32_t* __restrict__ offsets,
                                                     uint32_t n, uint64_t* __restrict__ status) {
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
        const uint64_t pre = lookback(chunks, chunk, total, status);
        if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint64_t o = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (i0 + k < m) tile_prefix[i0 + k] = (uint32_t)o;
        o += v[k];
    }
    if (chunk == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t nnz = s_prefix + total;
        offsets[n] = (uint32_t)nnz;
        status[0] = nnz;
    }
}

// Approximate join, step 3: offsets and ids of a warp tile from its stored
// entries and its prefix.
template <int PPT>
__global__ void __launch_bounds__(kJoinBlock) k_emit_approx(DevIndex X, uint32_t n, const uint64_t* __restrict__ entries,
                                                            const uint32_t* __restrict__ tile_prefix,
                                                            uint32_t* __restrict__ offsets, uint32_t* __restrict__ ids,
                                                            uint64_t ids_cap, uint64_t* __restrict__ status) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint64_t base = wt * (32 * PPT);
    if (base >= n) return;
    uint64_t e[PPT];
    uint32_t c[PPT], ex[PPT], run = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        e[k] = p < n ? __ldcs(entries + p) : 0ull;
        uint32_t nt, nc;
        entry_counts(X, e[k], &nt, &nc);
        c[k] = nt + nc;
        const uint32_t incl = warp_incl_scan(c[k]);
        ex[k] = run + incl - c[k];
        run += __shfl_sync(kFull, incl, 31);
    }
    const uint64_t prefix = tile_prefix[wt];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        if (p >= n) continue;
        const uint64_t o = prefix + ex[k];
        __stcs(offsets + p, (uint32_t)o);
        if (c[k]) {
            if (o + c[k] <= ids_cap) emit_all(X, e[k], ids, o);
            else atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrIdsCapacity);
        }
    }
}

// Exact join: number of output pairs of one point (true references plus the
// candidates that passed the PIP), -1 flags a corrupt queue position.
__device__ __forceinline__ uint32_t exact_count(const DevIndex& X, uint64_t e, const uint32_t* qbase, uint64_t p,
                                                const uint8_t* pass, uint64_t queue_cap, uint32_t* qb,
                                                uint64_t* status) {
    uint32_t nt, nc;
    entry_counts(X, e, &nt, &nc);
    *qb = 0;
    if (!nc) return nt;
    *qb = qbase[p];
    if ((uint64_t)*qb + nc > queue_cap) {   // cannot happen: the queue holds n * max_cand_refs
        atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrQueueOverflow);
        return 0xFFFFFFFFu;
    }
    uint32_t c = nt;
    for (uint32_t t = 0; t < nc; ++t) c += pass[*qb + t];
    return c;
}

template <int PPT>
__global__ void __launch_bounds__(kJoinBlock) k_emit_exact(DevIndex X, uint32_t n, const uint64_t* __restrict__ entries,
                                                           const uint32_t* __restrict__ qbase,
                                                           const uint8_t* __restrict__ pass, uint64_t queue_cap,
                                                           const uint32_t* __restrict__ tile_prefix,
                                                           uint32_t* __restrict__ offsets, uint32_t* __restrict__ ids,
                                                           uint64_t ids_cap, uint64_t* __restrict__ status) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint64_t base = wt * (32 * PPT);
    if (base >= n) return;
    uint64_t e[PPT];
    uint32_t cnt[PPT], qb[PPT], ex[PPT], run = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        e[k] = p < n ? entries[p] : 0ull;
        cnt[k] = p < n ? exact_count(X, e[k], qbase, p, pass, queue_cap, &qb[k], status) : 0u;
        if (cnt[k] == 0xFFFFFFFFu) { cnt[k] = 0; e[k] = 0; }
        const uint32_t incl = warp_incl_scan(cnt[k]);
        ex[k] = run + incl - cnt[k];
        run += __shfl_sync(kFull, incl, 31);
    }
    const uint64_t prefix = tile_prefix[wt];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        if (p >= n) continue;
        const uint64_t o = prefix + ex[k];
        __stcs(offsets + p, (uint32_t)o);
        if (!cnt[k]) continue;
        if (o + cnt[k] > ids_cap) {
            atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrIdsCapacity);
            continue;
        }
        const uint64_t ek = e[k];
        const uint32_t tag = (uint32_t)(ek & 3ull);
        uint64_t w = o;
        uint32_t ci = 0;
        if (tag == 1 || tag == 2) {
            for (int t = 0; t < (int)tag; ++t) {
                const uint32_t pl = payload_of(ek, t);
                if (pl & 1u) ids[w++] = pl >> 1;
                else if (pass[qb[k] + ci++]) ids[w++] = pl >> 1;
            }
        } else if (tag == 3) {
            const uint32_t off = payload_of(ek, 0);
            const uint32_t nt = __ldg(X.lut + off);
            const uint32_t* T = X.lut + off + 1;
            const uint32_t nc = __ldg(X.lut + off + 1 + nt);
            const uint32_t* Cc = X.lut + off + 2 + nt;
            uint32_t a = 0, b = 0;
            while (a < nt || b < nc) {
                const uint32_t ta = a < nt ? __ldg(T + a) : 0xFFFFFFFFu;
                const uint32_t cb = b < nc ? __ldg(Cc + b) : 0xFFFFFFFFu;
                if (ta < cb) { ids[w++] = ta; ++a; }
                else { if (pass[qb[k] + b]) ids[w++] = cb; ++b; }
            }
        }
    }
}

// Single CTA: exclusive scans of per-polygon candidate counts and chunk
// counts (chunks of kPipBlock candidates).
__global__ void __launch_bounds__(1024) k_poly_scan(const uint32_t* __restrict__ poly_count, uint32_t n_polys,
                                                    uint32_t* __restrict__ poly_start, uint32_t* __restrict__ cursor,
                                                    uint32_t* __restrict__ chunk_start, uint32_t* __restrict__ n_chunks) {
    __shared__ uint32_t s_warp[32];
    uint32_t carry_q = 0, carry_c = 0;
    for (uint32_t b = 0; b < n_polys; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t cnt = i < n_polys ? poly_count[i] : 0u;
        const uint32_t ch = (cnt + kPipBlock - 1) / kPipBlock;
        uint32_t tq, tc;
        const uint32_t eq = block_excl_scan<1024>(cnt, &tq, s_warp);
        const uint32_t ec = block_excl_scan<1024>(ch, &tc, s_warp);
        if (i < n_polys) {
            poly_start[i] = carry_q + eq;
            cursor[i] = carry_q + eq;
            chunk_start[i] = carry_c + ec;
        }
        carry_q += tq;
        carry_c += tc;
    }
    if (threadIdx.x == 0) {
        poly_start[n_polys] = carry_q;
        chunk_start[n_polys] = carry_c;
        *n_chunks = carry_c;
    }
}

// Groups the candidate queue by polygon (counting-sort scatter).  Each CTA
// takes chunks of kScatterChunk queue items, counts them per polygon with
// shared-memory atomics, reserves each polygon's slots with one global atomic
// per polygon and chunk, and writes the items' queue indices there.  With more
// polygons than shared counters, every item reserves its slot globally.
constexpr int kScatterChunk = 4096;
constexpr int kScatterMaxPolys = 4096;
__global__ void __launch_bounds__(256) k_scatter(const uint2* __restrict__ queue, const uint32_t* __restrict__ queue_len,
                                                 uint32_t* __restrict__ cursor, uint32_t* __restrict__ sorted,
                                                 uint64_t queue_cap, uint32_t n_polys) {
    __shared__ uint32_t s_cnt[kScatterMaxPolys];
    __shared__ uint32_t s_base[kScatterMaxPolys];
    const uint64_t len = min((uint64_t)*queue_len, queue_cap);
    if (n_polys > (uint32_t)kScatterMaxPolys) {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < len; q += stride) {
            const uint32_t pos = atomicAdd(&cursor[queue[q].y], 1u);
            sorted[pos] = (uint32_t)q;
        }
        return;
    }
    for (uint64_t c0 = (uint64_t)blockIdx.x * kScatterChunk; c0 < len; c0 += (uint64_t)gridDim.x * kScatterChunk) {
        const uint64_t c1 = min(c0 + kScatterChunk, len);
        for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x) s_cnt[p] = 0;
        __syncthreads();
        for (uint64_t q = c0 + threadIdx.x; q < c1; q += blockDim.x) atomicAdd(&s_cnt[queue[q].y], 1u);
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < n_polys; p += blockDim.x) {
            const uint32_t c = s_cnt[p];
            if (c) s_base[p] = atomicAdd(&cursor[p], c);
            s_cnt[p] = 0;
        }
        __syncthreads();
        for (uint64_t q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
            const uint32_t poly = queue[q].y;
            sorted[s_base[poly] + atomicAdd(&s_cnt[poly], 1u)] = (uint32_t)q;
        }
        __syncthreads();
    }
}

// ST_Covers in FP64 exactly as the spec (the certified test's fallback):
// same face, closed (u,v) bbox, ring rule with integer keys for the range
// tests and FP64 orientation, vertices read from global memory.
__device__ bool covers_fp64(const DevIndex& X, uint32_t poly, double lat, double lng) {
    if (!point_valid(lat, lng)) return false;
    double pu, pv;
    const int f = face_uv(lat, lng, &pu, &pv);
    if (f != X.poly_face[poly]) return false;
    const int64_t puk = dkey(pu), pvk = dkey(pv);
    const int64_t* bb = X.poly_bbox + 4ull * poly;
    if (!(puk >= bb[0] && puk <= bb[1] && pvk >= bb[2] && pvk <= bb[3])) return false;
    const uint32_t v0 = X.poly_off[poly], V = X.poly_off[poly + 1] - v0;
    bool inside = false;
    for (uint32_t k = 0; k < V; ++k) {
        const uint32_t a = v0 + k, b = v0 + (k + 1 == V ? 0u : k + 1);
        const int64_t av = X.poly_vkey[a], bv = X.poly_vkey[b];
        const int64_t vlo = av < bv ? av : bv, vhi = av < bv ? bv : av;
        if (pvk < vlo || pvk > vhi) continue;
        const double2 A = X.poly_uv[a], B = X.poly_uv[b];
        const double o = (B.x - A.x) * (pv - A.y) - (B.y - A.y) * (pu - A.x);
        if (o == 0.0) {
            const int64_t au = X.poly_ukey[a], bu = X.poly_ukey[b];
            if (puk >= (au < bu ? au : bu) && puk <= (au < bu ? bu : au)) return true;
        }
        if ((av <= pvk && pvk < bv && o > 0.0) || (bv <= pvk && pvk < av && o < 0.0)) inside = !inside;
    }
    return inside;
}

// Refine: ST_Covers of (point, polygon) candidates, grouped by polygon.  Per
// chunk of one polygon's candidates, the polygon's FP32 local vertices are
// staged in shared memory and every thread tests its candidate against the
// same edge at the same time (shared-memory broadcast).  The test is the
// certified FP32 one (covers_certified); an undecided candidate (within the
// error bounds of a vertex or an edge) is recomputed in FP64 (covers_fp64),
// as is every candidate of a polygon too large for the FP32 local frame.
__global__ void __launch_bounds__(kPipBlock) k_pip(DevIndex X, const double2* __restrict__ pts,
                                                   const uint2* __restrict__ queue, const uint32_t* __restrict__ sorted,
                                                   const uint32_t* __restrict__ poly_start,
                                                   const uint32_t* __restrict__ chunk_start,
                                                   const uint32_t* __restrict__ n_chunks, uint8_t* __restrict__ pass,
                                                   uint32_t* __restrict__ tile_count, uint64_t* __restrict__ undecided) {
    __shared__ F2 s_lv[kPipSmemVerts];
    const uint32_t total = *n_chunks;
    const uint32_t P = X.n_polys;
    uint32_t n_undecided = 0;
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        // polygon of chunk c: last poly with chunk_start <= c
        uint32_t lo = 0, hi = P;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (chunk_start[mid] <= c) lo = mid; else hi = mid;
        }
        const uint32_t poly = lo;
        const uint32_t q0 = poly_start[poly] + (c - chunk_start[poly]) * kPipBlock;
        const uint32_t q1 = min(q0 + kPipBlock, poly_start[poly + 1]);
        const uint32_t item = q0 + threadIdx.x;
        const uint32_t v0 = X.poly_off[poly], V = X.poly_off[poly + 1] - v0;
        const PolyLocal L = X.poly_local[poly];
        const bool certified = X.model.uv_enabled && L.ok && V <= (uint32_t)kPipSmemVerts;
        __syncthreads();
        if (certified)
            for (uint32_t t = threadIdx.x; t < V; t += blockDim.x) s_lv[t] = X.poly_luv[v0 + t];
        __syncthreads();
        if (item < q1) {
            const uint32_t qi = sorted[item];
            const uint2 qp = queue[qi];
            const double2 pt = pts[qp.x];
            int r = -1;
            float pu, pv, dp;
            if (certified && model_uv_local(X.model, pt.x, pt.y, L, &pu, &pv, &dp))
                r = covers_certified(s_lv, V, L, pu, pv, dp);
            if (r < 0) {
                r = covers_fp64(X, poly, pt.x, pt.y) ? 1 : 0;
                ++n_undecided;
            }
            pass[qi] = (uint8_t)r;
            if (r) atomicAdd(&tile_count[qp.x / kTile], 1u);
        }
    }
    warp_count(n_undecided, undecided);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

struct Layout {
    uint64_t hdr = 0, chunks = 0, pcount = 0, zero_end = 0;
    uint64_t entries = 0, tcount = 0, tprefix = 0;
    uint64_t qbase = 0, queue = 0, pass = 0, sorted = 0, pstart = 0, cursor = 0, cstart = 0, total = 0;
    uint64_t n_tiles = 0, n_chunks = 0, queue_cap = 0;
};

// scratch: [header 256 B: scan chunk counter u32, queue_len u32, n_chunks u32,
//           unused u32, FP64 cell-id fallbacks u64, FP64 refine fallbacks u64]
//          [scan chunk states] [exact: per-polygon candidate counts]
//          -- the part zeroed before every join --
//          [entries u64 per point] [tile counts u32] [tile prefixes u32]
//          then, exact mode only, the candidate queue and its polygon order
Layout layout(const Index& X, uint64_t n) {
    Layout L;
    L.n_tiles = (n + kTile - 1) / kTile;
    L.n_chunks = (L.n_tiles + 256 * kScanItems - 1) / (256 * kScanItems);
    uint64_t o = 256;
    L.chunks = o;
    o += align256(std::max<uint64_t>(L.n_chunks, 1) * 8);
    if (X.mode == AGJ_EXACT) {
        L.pcount = o;
        o += align256((uint64_t)X.n_polys * 4 + 4);
    }
    L.zero_end = o;
    L.entries = o; o += align256(n * 8 + 8);
    L.tcount = o; o += align256(L.n_tiles * 4 + 4);
    L.tprefix = o; o += align256(L.n_tiles * 4 + 4);
    if (X.mode == AGJ_EXACT) {
        const uint64_t P = X.n_polys;
        L.queue_cap = n * std::max<uint64_t>(X.stats.max_cand_refs, 1);
        L.qbase = o; o += align256(n * 4);
        L.queue = o; o += align256(L.queue_cap * 8);
        L.pass = o; o += align256(L.queue_cap);
        L.sorted = o; o += align256(L.queue_cap * 4);
        L.pstart = o; o += align256((P + 1) * 4);
        L.cursor = o; o += align256(P * 4 + 4);
        L.cstart = o; o += align256((P + 1) * 4);
    }
    L.total = o;
    return L;
}

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

}  // namespace

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
    if (cudaMalloc(&X->d_blob, o) != cudaSuccess) { cudaGetLastError(); X->d_blob = nullptr; return AGJ_ENOMEM; }
    if (cudaMemcpyAsync(X->d_blob, host.data(), o, cudaMemcpyHostToDevice, s) != cudaSuccess) return AGJ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AGJ_ECUDA;
    X->stats.device_bytes = o;
    cudaGetDevice(&X->device);
    return AGJ_OK;
}

int join_requirements(const Index& X, uint64_t n, agj_requirements* r) {
    const Layout L = layout(X, n);
    r->ids_capacity = n * std::max<uint64_t>(X.stats.max_refs, 1);
    r->scratch_bytes = L.total;
    return AGJ_OK;
}

int launch_cell_ids(const double* d_points, uint64_t n, uint64_t* d_ids, cudaStream_t s) {
    if (n == 0) return AGJ_OK;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sm_count() * 16);
    k_cell_ids<<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(d_points), n, d_ids);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

int launch_join(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, agj_pairs* out,
                cudaEvent_t const* events) {
    auto mark = [&](int k) {
        if (events) cudaEventRecord(events[k], s);
    };
    if (!out || !out->offsets || !out->status || (n && !d_points)) return AGJ_EINVAL;
    if (n >= 0xFFFFFFFFull) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return AGJ_EINVAL;
    const Layout L = layout(X, n);
    agj_requirements req;
    join_requirements(X, n, &req);
    if (req.ids_capacity >= 0xFFFFFFFFull) return AGJ_ECAPACITY;    // offsets are 32-bit: split the batch
    if (!out->scratch || out->scratch_bytes < L.total || out->ids_capacity < req.ids_capacity ||
        (req.ids_capacity && !out->ids) || (reinterpret_cast<uintptr_t>(out->scratch) & 255u) != 0)
        return AGJ_ECAPACITY;
    char* sc = static_cast<char*>(out->scratch);
    const DevIndex D = make_dev_index(X);
    const double2* pts = reinterpret_cast<const double2*>(d_points);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sc);
    uint64_t* fallbacks = reinterpret_cast<uint64_t*>(sc) + 2;
    uint64_t* chunks = reinterpret_cast<uint64_t*>(sc + L.chunks);
    uint64_t* entries = reinterpret_cast<uint64_t*>(sc + L.entries);
    uint32_t* tcount = reinterpret_cast<uint32_t*>(sc + L.tcount);
    uint32_t* tprefix = reinterpret_cast<uint32_t*>(sc + L.tprefix);
    // zero the header, the scan chunk states (and polygon counts) and the status words
    {
        const uint64_t zero_words = L.zero_end / 8;
        const int grid = (int)std::min<uint64_t>((zero_words + 255) / 256 + 1, (uint64_t)sm_count() * 4);
        k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), zero_words, out->status, 4);
    }
    if (n == 0) {
        cudaMemsetAsync(out->offsets, 0, 4, s);
        for (int k = 0; k < 4; ++k) mark(k);
        return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    }
    const unsigned grid = (unsigned)((L.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
    mark(0);
    if (X.mode == AGJ_APPROX) {
        k_probe_approx<kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, pts, (uint32_t)n, entries, tcount, out->status, fallbacks);
        mark(1);
        k_scan_counts<<<(unsigned)L.n_chunks, 256, 0, s>>>(tcount, L.n_tiles, tprefix, chunks, hdr, out->offsets,
                                                           (uint32_t)n, out->status);
        mark(2);
        k_emit_approx<kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, (uint32_t)n, entries, tprefix, out->offsets, out->ids,
                                                            out->ids_capacity, out->status);
        mark(3);
    } else {
        uint32_t* qbase = reinterpret_cast<uint32_t*>(sc + L.qbase);
        uint2* queue = reinterpret_cast<uint2*>(sc + L.queue);
        uint8_t* pass = reinterpret_cast<uint8_t*>(sc + L.pass);
        uint32_t* sorted = reinterpret_cast<uint32_t*>(sc + L.sorted);
        uint32_t* pcount = reinterpret_cast<uint32_t*>(sc + L.pcount);
        uint32_t* pstart = reinterpret_cast<uint32_t*>(sc + L.pstart);
        uint32_t* cursor = reinterpret_cast<uint32_t*>(sc + L.cursor);
        uint32_t* cstart = reinterpret_cast<uint32_t*>(sc + L.cstart);
        k_probe_exact<kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, pts, (uint32_t)n, entries, qbase, queue, L.queue_cap,
                                                            hdr + 1, pcount, tcount, out->status, fallbacks);
        mark(1);
        if (X.n_polys) {
            k_poly_scan<<<1, 1024, 0, s>>>(pcount, X.n_polys, pstart, cursor, cstart, hdr + 2);
            const int sgrid = sm_count() * 4;
            k_scatter<<<sgrid, 256, 0, s>>>(queue, hdr + 1, cursor, sorted, L.queue_cap, X.n_polys);
            k_pip<<<sm_count() * 4, kPipBlock, 0, s>>>(D, pts, queue, sorted, pstart, cstart, hdr + 2, pass, tcount,
                                                        reinterpret_cast<uint64_t*>(sc) + 3);
        }
        mark(2);
        k_scan_counts<<<(unsigned)L.n_chunks, 256, 0, s>>>(tcount, L.n_tiles, tprefix, chunks, hdr, out->offsets,
                                                           (uint32_t)n, out->status);
        k_emit_exact<kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, (uint32_t)n, entries, qbase, pass, L.queue_cap, tprefix,
                                                           out->offsets, out->ids, out->ids_capacity, out->status);
        mark(3);
    }
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
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
        D, reinterpret_cast<const double2*>(d_points), (uint32_t)n, d_offsets, d_ids, ids_capacity,
        sc + kNoAllocHeaderWords, reinterpret_cast<uint32_t*>(sc), d_status, sc + 2);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

}  // namespace agj
