// agj_kernels.cu — sm_103a kernels of the probe side (§III-E) and their
// launchers.
//
//   k_cell_ids       point -> 64-bit cell id (FP64 spec of agj_geom.cuh)
//   k_join_approx    one pass per tile: cell id, face/prefix stage, trie walk
//                    (Listing "Probe Adaptive Cell Trie"), entry decode, tile
//                    scan with decoupled look-back, CSR write (approximate
//                    join: every reference is output, §V "approx")
//   k_probe_exact    cell id + walk + decode; true hits counted, candidate
//                    references compacted by warp ballot into a queue
//   k_poly_scan      per-polygon candidate counts -> queue segments + chunks
//   k_scatter        queue grouped by polygon
//   k_pip            exact ST_Covers refine (§II "PIP"): one CTA per chunk of
//                    one polygon's candidates, the polygon's edges staged in
//                    shared memory and read by all threads (broadcast)
//   k_csr_exact      true hits + passing candidates -> CSR (one pass, look-back)
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
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kJoinBlock = 256;
constexpr int kJoinPPT = 4;
constexpr int kTile = kJoinBlock * kJoinPPT;
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
// per-tile point staging + walk
// ---------------------------------------------------------------------------

// Cell ids and trie entries for PPT consecutive points per thread; walks of
// the PPT points advance level by level together so their gathers overlap.
template <int PPT>
__device__ __forceinline__ uint32_t probe_points(const DevIndex& X, const DevFace* faces, const double2* s_pts, int first,
                                                 int valid, uint64_t e[PPT], uint64_t* err) {
    uint32_t gathers = 0;
    uint64_t key[PPT];
    const uint64_t* node[PPT];
    bool act[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        e[k] = 0;
        act[k] = false;
        node[k] = X.nodes;
        key[k] = 0;
        if (k < valid) {
            const double2 p = s_pts[first + k];
            const uint64_t id = point_cell_id(p.x, p.y);
            if (id != kInvalidId) {
                const DevFace fr = faces[id >> 61];
                if (fr.root != kNoRootDev) {
                    uint64_t kk = id << 3;
                    bool ok = true;
                    if (fr.prefix_bits) {
                        ok = (kk >> (64 - fr.prefix_bits)) == fr.prefix;
                        kk <<= fr.prefix_bits;
                    }
                    if (ok) {
                        act[k] = true;
                        key[k] = kk;
                        node[k] = X.nodes + (uint64_t)fr.root * 256;
                    }
                }
            }
        }
    }
    const char* base = reinterpret_cast<const char*>(X.nodes);
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        uint64_t v[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) v[k] = act[k] ? __ldg(node[k] + (key[k] >> 56)) : 0ull;
#pragma unroll
        for (int k = 0; k < PPT; ++k) gathers += act[k] ? 1u : 0u;
        bool any = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (!act[k]) continue;
            key[k] <<= 8;
            if ((v[k] & 3ull) != 0ull || v[k] == 0ull) {
                e[k] = v[k];
                act[k] = false;
            } else if ((v[k] >> 11) >= X.n_nodes) {
                atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
                act[k] = false;
            } else {
                node[k] = reinterpret_cast<const uint64_t*>(base + v[k]);
                any = true;
            }
        }
        if (!any) break;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        if (act[k]) {
            atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
            e[k] = 0;
        }
    return gathers;
}

// Adds a per-thread count to a device counter with one atomic per warp.
__device__ __forceinline__ void warp_count(uint32_t v, uint64_t* counter) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)counter, (unsigned long long)v);
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

template <int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK) k_join_approx(DevIndex X, const double2* __restrict__ pts, uint32_t n,
                                                       uint32_t* __restrict__ offsets, uint32_t* __restrict__ ids,
                                                       uint64_t ids_cap, uint64_t* __restrict__ tiles,
                                                       uint32_t* __restrict__ tile_counter, uint64_t* __restrict__ status) {
    constexpr int TILE = BLOCK * PPT;
    __shared__ DevFace s_faces[6];
    __shared__ double2 s_pts[TILE];
    __shared__ uint32_t s_warp[BLOCK / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x < 6) s_faces[threadIdx.x] = X.faces[threadIdx.x];
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t tbase = (uint64_t)tile * TILE;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = tbase + (uint64_t)k * BLOCK + threadIdx.x;
        if (p < n) s_pts[k * BLOCK + threadIdx.x] = pts[p];
    }
    __syncthreads();
    const uint64_t my0 = tbase + (uint64_t)threadIdx.x * PPT;
    const int valid = my0 >= n ? 0 : (int)min((uint64_t)PPT, n - my0);
    uint64_t e[PPT];
    warp_count(probe_points<PPT>(X, s_faces, s_pts, threadIdx.x * PPT, valid, e, &status[1]), &status[3]);
    uint32_t c[PPT], sum = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt, nc;
        entry_counts(X, e[k], &nt, &nc);
        c[k] = nt + nc;
        sum += c[k];
    }
    uint32_t block_total;
    const uint32_t excl = block_excl_scan<BLOCK>(sum, &block_total, s_warp);
    if (threadIdx.x < 32) {
        const uint64_t pre = lookback(tiles, tile, block_total, status);
        if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint64_t o = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (k < valid) {
            offsets[my0 + k] = (uint32_t)o;
            if (c[k]) {
                if (o + c[k] <= ids_cap) emit_all(X, e[k], ids, o);
                else atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrIdsCapacity);
            }
            o += c[k];
        }
    }
    if (tile == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t nnz = s_prefix + block_total;
        offsets[n] = (uint32_t)nnz;
        status[0] = nnz;
    }
}

// Exact-mode probe: entries + compacted candidate queue.
template <int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK) k_probe_exact(DevIndex X, const double2* __restrict__ pts, uint32_t n,
                                                       uint64_t* __restrict__ entries, uint32_t* __restrict__ qbase,
                                                       uint2* __restrict__ queue, uint64_t queue_cap,
                                                       uint32_t* __restrict__ queue_len,
                                                       uint32_t* __restrict__ poly_count, uint64_t* __restrict__ status) {
    constexpr int TILE = BLOCK * PPT;
    __shared__ DevFace s_faces[6];
    __shared__ double2 s_pts[TILE];
    if (threadIdx.x < 6) s_faces[threadIdx.x] = X.faces[threadIdx.x];
    const uint64_t tbase = (uint64_t)blockIdx.x * TILE;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = tbase + (uint64_t)k * BLOCK + threadIdx.x;
        if (p < n) s_pts[k * BLOCK + threadIdx.x] = pts[p];
    }
    __syncthreads();
    const uint64_t my0 = tbase + (uint64_t)threadIdx.x * PPT;
    const int valid = my0 >= n ? 0 : (int)min((uint64_t)PPT, n - my0);
    uint64_t e[PPT];
    warp_count(probe_points<PPT>(X, s_faces, s_pts, threadIdx.x * PPT, valid, e, &status[1]), &status[3]);
    uint32_t nc[PPT], csum = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt;
        entry_counts(X, e[k], &nt, &nc[k]);
        csum += nc[k];
        if (k < valid) entries[my0 + k] = e[k];
    }
    // warp-ballot compaction: one atomic per warp reserves the warp's slots
    const int lane = threadIdx.x & 31;
    uint32_t x = csum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const uint32_t wtotal = __shfl_sync(kFull, x, 31);
    if (__ballot_sync(kFull, csum != 0) == 0) return;
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
        const uint32_t p = (uint32_t)(my0 + k);
        qbase[p] = (uint32_t)q;
        const uint64_t ek = e[k];
        const uint32_t tag = (uint32_t)(ek & 3ull);
        uint32_t polys[2];
        uint32_t m = 0;
        if (tag == 1 || tag == 2) {
            for (int w = 0; w < (int)tag; ++w) {
                const uint32_t pl = payload_of(ek, w);
                if (!(pl & 1u)) polys[m++] = pl >> 1;
            }
            for (uint32_t t = 0; t < m; ++t) {
                if (q < queue_cap) { queue[q] = make_uint2(p, polys[t]); atomicAdd(&poly_count[polys[t]], 1u); }
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

__global__ void k_scatter(const uint2* __restrict__ queue, const uint32_t* __restrict__ queue_len,
                          uint32_t* __restrict__ cursor, uint32_t* __restrict__ sorted, uint64_t queue_cap) {
    const uint64_t len = min((uint64_t)*queue_len, queue_cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < len; q += stride) {
        const uint32_t pos = atomicAdd(&cursor[queue[q].y], 1u);
        sorted[pos] = (uint32_t)q;
    }
}

// Refine: ST_Covers of (point, polygon) candidates, grouped by polygon.
// Per chunk the polygon's vertices (u,v), and the integer keys of their u
// and v, are staged in shared memory; every thread tests its candidate
// against the same edge at the same time (shared-memory broadcast).  Edges
// whose v-range misses the point are skipped with integer compares; only
// edges straddling the point's v use FP64 (the orientation of the ring rule).
__global__ void __launch_bounds__(kPipBlock) k_pip(DevIndex X, const double2* __restrict__ pts,
                                                   const uint2* __restrict__ queue, const uint32_t* __restrict__ sorted,
                                                   const uint32_t* __restrict__ poly_start,
                                                   const uint32_t* __restrict__ chunk_start,
                                                   const uint32_t* __restrict__ n_chunks, uint8_t* __restrict__ pass) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2* s_uv = reinterpret_cast<double2*>(smem);
    int64_t* s_vk = reinterpret_cast<int64_t*>(smem + sizeof(double2) * (kPipSmemVerts + 1));
    int64_t* s_uk = s_vk + (kPipSmemVerts + 1);
    const uint32_t total = *n_chunks;
    const uint32_t P = X.n_polys;
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
        const bool have = item < q1;
        uint32_t qi = 0;
        double pu = 0, pv = 0;
        int64_t puk = 0, pvk = 0;
        bool alive = false;
        const uint32_t v0 = X.poly_off[poly], V = X.poly_off[poly + 1] - v0;
        if (have) {
            qi = sorted[item];
            const uint2 qp = queue[qi];
            const double2 pt = pts[qp.x];
            if (point_valid(pt.x, pt.y)) {
                const int f = face_uv(pt.x, pt.y, &pu, &pv);
                puk = dkey(pu);
                pvk = dkey(pv);
                const int64_t* bb = X.poly_bbox + 4ull * poly;
                alive = f == X.poly_face[poly] && puk >= bb[0] && puk <= bb[1] && pvk >= bb[2] && pvk <= bb[3];
            }
        }
        bool inside = false, on_edge = false;
        for (uint32_t s = 0; s < V; s += kPipSmemVerts) {
            const uint32_t m = min((uint32_t)kPipSmemVerts, V - s);   // edges s .. s+m-1
            __syncthreads();
            for (uint32_t t = threadIdx.x; t <= m; t += blockDim.x) {
                const uint32_t g = v0 + ((s + t) == V ? 0u : (s + t));
                s_uv[t] = X.poly_uv[g];
                s_vk[t] = X.poly_vkey[g];
                s_uk[t] = X.poly_ukey[g];
            }
            __syncthreads();
            if (__syncthreads_or(alive)) {
                if (alive) {
                    for (uint32_t k = 0; k < m; ++k) {
                        const int64_t av = s_vk[k], bv = s_vk[k + 1];
                        const int64_t vlo = av < bv ? av : bv, vhi = av < bv ? bv : av;
                        if (pvk < vlo || pvk > vhi) continue;
                        const double2 A = s_uv[k], B = s_uv[k + 1];
                        const double o = (B.x - A.x) * (pv - A.y) - (B.y - A.y) * (pu - A.x);
                        if (o == 0.0) {
                            const int64_t au = s_uk[k], bu = s_uk[k + 1];
                            if (puk >= (au < bu ? au : bu) && puk <= (au < bu ? bu : au)) on_edge = true;
                        }
                        if ((av <= pvk && pvk < bv && o > 0.0) || (bv <= pvk && pvk < av && o < 0.0)) inside = !inside;
                    }
                }
            }
        }
        if (have) pass[qi] = (uint8_t)(alive && (on_edge || inside));
    }
}

template <int BLOCK, int PPT>
__global__ void __launch_bounds__(BLOCK) k_csr_exact(DevIndex X, uint32_t n, const uint64_t* __restrict__ entries,
                                                     const uint32_t* __restrict__ qbase, const uint8_t* __restrict__ pass,
                                                     uint64_t queue_cap,
                                                     uint32_t* __restrict__ offsets, uint32_t* __restrict__ ids,
                                                     uint64_t ids_cap, uint64_t* __restrict__ tiles,
                                                     uint32_t* __restrict__ tile_counter, uint64_t* __restrict__ status) {
    constexpr int TILE = BLOCK * PPT;
    __shared__ uint32_t s_warp[BLOCK / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t my0 = (uint64_t)tile * TILE + (uint64_t)threadIdx.x * PPT;
    const int valid = my0 >= n ? 0 : (int)min((uint64_t)PPT, n - my0);
    uint64_t e[PPT];
    uint32_t cnt[PPT], qb[PPT], sum = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        e[k] = k < valid ? entries[my0 + k] : 0ull;
        uint32_t nt, nc;
        entry_counts(X, e[k], &nt, &nc);
        cnt[k] = nt;
        qb[k] = 0;
        if (nc) {
            qb[k] = qbase[my0 + k];
            if ((uint64_t)qb[k] + nc > queue_cap) {   // cannot happen: the queue holds n * max_cand_refs
                atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrQueueOverflow);
                e[k] = 0;
                nc = 0;
            }
            for (uint32_t t = 0; t < nc; ++t) cnt[k] += pass[qb[k] + t];
        }
        sum += cnt[k];
    }
    uint32_t block_total;
    const uint32_t excl = block_excl_scan<BLOCK>(sum, &block_total, s_warp);
    if (threadIdx.x < 32) {
        const uint64_t pre = lookback(tiles, tile, block_total, status);
        if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint64_t o = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (k >= valid) continue;
        offsets[my0 + k] = (uint32_t)o;
        if (!cnt[k]) continue;
        if (o + cnt[k] > ids_cap) {
            atomicOr((unsigned long long*)&status[1], (unsigned long long)kErrIdsCapacity);
            o += cnt[k];
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
        o += cnt[k];
    }
    if (tile == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t nnz = s_prefix + block_total;
        offsets[n] = (uint32_t)nnz;
        status[0] = nnz;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

struct Layout {
    uint64_t hdr = 0, tiles = 0, entries = 0, qbase = 0, queue = 0, pass = 0, sorted = 0;
    uint64_t pcount = 0, pstart = 0, cursor = 0, cstart = 0, total = 0;
    uint64_t n_tiles = 0, queue_cap = 0;
};

// scratch: [header 256 B: tile counter u32, queue_len u32, n_chunks u32]
//          [tile states] [exact: per-polygon candidate counts] -- the part
//          zeroed before every join -- then, exact mode only, the candidate
//          queue and its polygon-grouped order
Layout layout(const Index& X, uint64_t n) {
    Layout L;
    L.n_tiles = (n + kTile - 1) / kTile;
    uint64_t o = 256;
    L.tiles = o;
    o += align256(std::max<uint64_t>(L.n_tiles, 1) * 8);
    if (X.mode == AGJ_EXACT) {
        const uint64_t P = X.n_polys;
        L.pcount = o; o += align256(P * 4 + 4);
        L.hdr = o;   // end of the zeroed prefix
        L.queue_cap = n * std::max<uint64_t>(X.stats.max_cand_refs, 1);
        L.entries = o; o += align256(n * 8);
        L.qbase = o; o += align256(n * 4);
        L.queue = o; o += align256(L.queue_cap * 8);
        L.pass = o; o += align256(L.queue_cap);
        L.sorted = o; o += align256(L.queue_cap * 4);
        L.pstart = o; o += align256((P + 1) * 4);
        L.cursor = o; o += align256(P * 4 + 4);
        L.cstart = o; o += align256((P + 1) * 4);
    } else {
        L.hdr = o;
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
    D.n_nodes = X.nodes.size() / 256;
    D.n_lut = X.lut.size();
    D.n_polys = X.n_polys;
    D.max_depth = X.stats.max_depth;
    for (int f = 0; f < 6; ++f) D.faces[f] = DevFace{X.faces[f].root, X.faces[f].prefix_bits, X.faces[f].prefix};
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

int launch_join(const Index& X, const double* d_points, uint64_t n, cudaStream_t s, agj_pairs* out) {
    if (!out || !out->offsets || !out->status || (n && !d_points)) return AGJ_EINVAL;
    if (n >= 0xFFFFFFFFull) return AGJ_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_points) & 15u) != 0) return AGJ_EINVAL;
    const Layout L = layout(X, n);
    agj_requirements req;
    join_requirements(X, n, &req);
    if (!out->scratch || out->scratch_bytes < L.total || out->ids_capacity < req.ids_capacity ||
        (req.ids_capacity && !out->ids) || (reinterpret_cast<uintptr_t>(out->scratch) & 255u) != 0)
        return AGJ_ECAPACITY;
    char* sc = static_cast<char*>(out->scratch);
    const DevIndex D = make_dev_index(X);
    const double2* pts = reinterpret_cast<const double2*>(d_points);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sc);
    uint64_t* tiles = reinterpret_cast<uint64_t*>(sc + L.tiles);
    // zero the header + tile states (+ polygon counts) and the status words
    const uint64_t zero_words = L.hdr / 8;
    {
        const int grid = (int)std::min<uint64_t>((zero_words + 255) / 256 + 1, (uint64_t)sm_count() * 4);
        k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), zero_words, out->status, 4);
    }
    if (n == 0) {
        cudaMemsetAsync(out->offsets, 0, 4, s);
        return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
    }
    const unsigned grid = (unsigned)L.n_tiles;
    if (X.mode == AGJ_APPROX) {
        k_join_approx<kJoinBlock, kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, pts, (uint32_t)n, out->offsets, out->ids,
                                                                      out->ids_capacity, tiles, hdr, out->status);
    } else {
        uint64_t* entries = reinterpret_cast<uint64_t*>(sc + L.entries);
        uint32_t* qbase = reinterpret_cast<uint32_t*>(sc + L.qbase);
        uint2* queue = reinterpret_cast<uint2*>(sc + L.queue);
        uint8_t* pass = reinterpret_cast<uint8_t*>(sc + L.pass);
        uint32_t* sorted = reinterpret_cast<uint32_t*>(sc + L.sorted);
        uint32_t* pcount = reinterpret_cast<uint32_t*>(sc + L.pcount);
        uint32_t* pstart = reinterpret_cast<uint32_t*>(sc + L.pstart);
        uint32_t* cursor = reinterpret_cast<uint32_t*>(sc + L.cursor);
        uint32_t* cstart = reinterpret_cast<uint32_t*>(sc + L.cstart);
        k_probe_exact<kJoinBlock, kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, pts, (uint32_t)n, entries, qbase, queue,
                                                                      L.queue_cap, hdr + 1, pcount, out->status);
        if (X.n_polys) {
            k_poly_scan<<<1, 1024, 0, s>>>(pcount, X.n_polys, pstart, cursor, cstart, hdr + 2);
            const int sgrid = sm_count() * 4;
            k_scatter<<<sgrid, 256, 0, s>>>(queue, hdr + 1, cursor, sorted, L.queue_cap);
            const size_t smem = (sizeof(double2) + 16) * (kPipSmemVerts + 1);
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_pip, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                attr = true;
            }
            k_pip<<<sm_count() * 2, kPipBlock, smem, s>>>(D, pts, queue, sorted, pstart, cstart, hdr + 2, pass);
        }
        k_csr_exact<kJoinBlock, kJoinPPT><<<grid, kJoinBlock, 0, s>>>(D, (uint32_t)n, entries, qbase, pass,
                                                                     L.queue_cap, out->offsets, out->ids, out->ids_capacity, tiles,
                                                                     hdr, out->status);
    }
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

// ---------------------------------------------------------------------------
// approximate join without any allocation
// ---------------------------------------------------------------------------
// The one-pass approximate join needs work space for its tile scan: a
// 256-byte header (the tile counter) and one 8-byte state per tile of
// kTile points.  For callers that must not allocate, that work space is this
// file-scope device array, sized for joins of up to kNoAllocMaxPoints points
// (16384 tiles, 128 KiB + 256 B).  Every device that loads the library holds
// one copy until the process exits.  All calls on a device share it, so
// calls whose kernels overlap on the GPU race; the header and the tile
// states a call uses are cleared at the start of every call.
constexpr uint64_t kNoAllocMaxPoints = 1ull << 24;
constexpr uint64_t kNoAllocHeaderWords = 32;
constexpr uint64_t kNoAllocTiles = kNoAllocMaxPoints / kTile;
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
    const uint64_t n_tiles = (n + kTile - 1) / kTile;
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
    k_join_approx<kJoinBlock, kJoinPPT><<<(unsigned)n_tiles, kJoinBlock, 0, s>>>(
        D, reinterpret_cast<const double2*>(d_points), (uint32_t)n, d_offsets, d_ids, ids_capacity,
        sc + kNoAllocHeaderWords, reinterpret_cast<uint32_t*>(sc), d_status);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

}  // namespace agj
