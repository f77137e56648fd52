// agj_probe.cuh — device side of the join, shared by the plain join
// (agj_kernels.cu) and the batched form (agj_batch.cu): the per-point probe
// (cell id, face/prefix stage, trie walk, entry decode), scans, the refine
// test, and the join kernels, templated on the points per lane (PPT) and on
// the job source:
//   OneJob    the plain join: one job descriptor passed by value;
//   ManyJobs  the batched form: an array of job descriptors whose points and
//             polygons are laid end to end in a global tile and polygon
//             space; a tile or polygon finds its job by binary search.
// Kernels iterate over global warp tiles with a grid stride, so the same code
// runs as one CTA per tile group (plain join) or as a persistent grid
// (batched form).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "agj_device.cuh"
#include "agj_geom.cuh"

namespace agj {

constexpr uint32_t kFull = 0xFFFFFFFFu;
// The walk's Hilbert table: the 4-level table of make_hilbert_lut with each
// entry rearranged to (next orientation << 9) | position byte: the next row's
// byte offset in the table and the key byte are one mask each.
constexpr HilbertLut make_walk_lut() {
    HilbertLut H = make_hilbert_lut(), W{};
    for (uint32_t idx = 0; idx < 1024; ++idx) W.v[idx] = (uint16_t)(((H.v[idx] & 3u) << 9) | (H.v[idx] >> 2));
    return W;
}
static __device__ __align__(16) const HilbertLut g_hilbert_lut = make_walk_lut();
constexpr uint32_t kSpinLimit = 1u << 22;
// Resident CTAs per SM the probe kernels are compiled for (a register cap:
// 65536 / (256 x blocks) per thread).  The probe is latency-bound (dependent
// trie gathers), so more resident warps pay while the registers last: at 5
// CTAs (40 warps, 48 registers) the probes, single-job and batched, need no
// spills and beat 4 CTAs on the city workload; at 6 (40 registers) the walk
// spills.  A plain join of kJoinWidePoints points or more runs 4 points per
// lane: its approximate probe at 4 CTAs (64 registers, 32 warps = 4096
// walks per SM), its exact probe at 5 (48 registers; a few spilled bytes
// cost less than the lost warps).
#ifndef AGJ_PROBE_MIN_BLOCKS
#define AGJ_PROBE_MIN_BLOCKS 5
#endif
#ifndef AGJ_JOIN_APPROX_PROBE_MIN_BLOCKS
#define AGJ_JOIN_APPROX_PROBE_MIN_BLOCKS 4
#endif
#ifndef AGJ_BATCH_PROBE_MIN_BLOCKS
#define AGJ_BATCH_PROBE_MIN_BLOCKS 5
#endif
#ifndef AGJ_APPROX_PROBE_MIN_BLOCKS
#define AGJ_APPROX_PROBE_MIN_BLOCKS 5
#endif
// Each CTA of the plain join's probe prefetches into the L2 the points of
// the CTA one grid of resident CTAs ahead (1) or not (0).
// The plain join's probe waits for its CTA's shared tables on a
// tables-ready mbarrier (1) or on a CTA barrier after the cell ids (0).
#ifndef AGJ_PROBE_READY_BARRIER
#define AGJ_PROBE_READY_BARRIER 1
#endif
#ifndef AGJ_PREFETCH_AHEAD
#define AGJ_PREFETCH_AHEAD 1
#endif
constexpr int kJoinBlock = 256;
// Points per lane.  A wide plain join (kJoinWidePoints and more) takes 4:
// fewer tiles, more walks in flight per warp.  A smaller join takes 2, which
// spreads its few points over twice the warps (below a few resident waves
// the probe's time is the slowest warp's walk, 11.0 against 13.8 us per
// 1e5-point join); so do the count(*) aggregation, whose per-point
// histogram work makes the wider tile slower (58.0 against 51.6 G points/s
// on the city workload), and the training pass.
constexpr int kJoinPPT = 4;
constexpr int kJoinSmallPPT = 2;
constexpr uint64_t kJoinWidePoints = 1ull << 21;
constexpr int kWarpsPerBlock = kJoinBlock / 32;
constexpr int kPipBlock = 256;
constexpr int kPipSmemVerts = 2048;            // vertices staged per CTA (8 B each)
constexpr int kScanItems = 16;

// ---------------------------------------------------------------------------
// scans
// ---------------------------------------------------------------------------

template <int BLOCK, class T>
__device__ __forceinline__ T block_excl_scan(T v, T* total, T* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = BLOCK / 32;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    *total = s_warp[NW - 1];
    const T wp = warp ? s_warp[warp - 1] : T(0);
    __syncthreads();
    return wp + x - v;
}

// Decoupled look-back across tiles (run by one full warp).  Tile states are
// 64-bit words: top 2 bits 0 = not ready, 1 = aggregate, 2 = inclusive
// prefix; low 62 bits the value.  Tiles are numbered in the order their CTAs
// started (atomic counter), so every predecessor is running or done and the
// wait ends; it is bounded all the same and sets kErrScanTimeout in *err.
__device__ __forceinline__ uint64_t lookback(uint64_t* tiles, uint32_t tile, uint64_t total, uint64_t* err) {
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
                    atomicOr((unsigned long long*)err, (unsigned long long)kErrScanTimeout);
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
    uint32_t i32, j32;      // (i, j) << (2 + 4 b): the next byte's 4 levels on top; 0 padding below
    uint32_t o;             // Hilbert orientation before byte b, << 9 (its row's byte offset in the table)
    uint32_t node;          // current trie node
    int32_t left;           // certified key bytes left, from byte b on
    int32_t st;             // 0 done, 1 walking, 2 needs the FP64 cell id
};

// The next key byte (levels 4b+1 .. 4b+4) from the walk's Hilbert table.
__device__ __forceinline__ uint32_t next_byte(const uint16_t* lut, Walk& w) {
    const uint32_t off = w.o | ((w.i32 >> 23) & 0x1E0u) | ((w.j32 >> 27) & 0x1Eu);
    const uint32_t t = *reinterpret_cast<const uint16_t*>(reinterpret_cast<const char*>(lut) + off);
    w.i32 <<= 4;
    w.j32 <<= 4;
    w.o = t & 0x600u;
    --w.left;
    return t & 0xFFu;
}

// Leaf cell of a point: face, (i, j) and the leading levels certified.
struct PointIJ {
    uint32_t i, j;
    int lc, face;
};

// Cell id stage (§IV-B stage 1) for one point.  With the index's fast model
// (and exact == false) the id comes from the certified FP32 path; otherwise
// from the FP64 spec.  Returns false when the point lies in no cell (invalid,
// or outside the fast model's window).
__device__ __forceinline__ bool point_ij(const FastModel& M, double lat, double lng, bool exact, PointIJ& p) {
    if (!exact && M.enabled) {
        if (!model_ij(M, lat, lng, &p.i, &p.j, &p.lc)) return false;   // outside the window: in no cell
        p.face = M.face;
        if (p.lc >= kLevels) p.lc = kLevels + 2;                            // exact id: padding levels too
        return true;
    }
    if (!point_valid(lat, lng)) return false;
    double u, v;
    p.face = face_uv(lat, lng, &u, &v);
    p.i = st_to_ij(uv_to_st(u));
    p.j = st_to_ij(uv_to_st(v));
    p.lc = kLevels + 2;
    return true;
}

// Face/prefix stage (§IV-B stage 1) for one point's leaf cell.  Leaves
// w.st = 0 when the point joins nothing, 1 when the walk can start at
// w.node, 2 when an uncertified level decides the prefix.  The prefix is
// compared as a cell (its level-30 bounds in i and j), which equals
// comparing the key's prefix bytes; the walk then starts at the prefix's
// orientation with the next key byte.
__device__ __forceinline__ void start_walk(const DevFace* faces, const uint16_t*, const PointIJ& p, Walk& w) {
    w.st = 0;
    w.o = 0;
    const DevFace fr = faces[p.face];
    if (fr.root == kNoRootDev) return;
    const int32_t nb = (int32_t)(fr.prefix_bits >> 3);
    const int32_t left = (p.lc >> 2) - nb;
    if (left < 0) { w.st = 2; return; }
    if (((p.i ^ fr.pi) | (p.j ^ fr.pj)) & fr.pmask) return;
    const uint32_t sh = 2u + 4u * (uint32_t)nb;
    w.i32 = p.i << sh;
    w.j32 = p.j << sh;
    w.o = fr.o_row;
    w.left = left;
    w.node = fr.root;
    w.st = 1;
}

__device__ __forceinline__ void begin_walk(const DevIndex& X, const DevFace* faces, const uint16_t* lut, double lat,
                                           double lng, bool exact, Walk& w) {
    PointIJ p;
    w.st = 0;
    w.o = 0;
    if (point_ij(X.model, lat, lng, exact, p)) start_walk(faces, lut, p, w);
}

// Trie levels every walk of a warp takes in step before the unfinished ones
// are compacted (root + two levels: nearly every walk of the city-scale
// indexes needs them, about one in eight needs more).
#ifndef AGJ_LOCK_LEVELS
#define AGJ_LOCK_LEVELS 3
#endif
constexpr int kLockLevels = AGJ_LOCK_LEVELS;

// One level of a walk (Listing "Probe Adaptive Cell Trie"), without
// branches: a live walk whose next key byte is certified reads that byte's
// entry (from the shared copy of the root with kRoot) into v and either
// descends or ends there; one whose next byte is not certified is marked
// for the FP64 id (st 2).  v keeps the last entry read, which is the walk's
// result once it ends.  Finished walks step along harmlessly (their key
// state is not used again).  Child entries hold node << 11 with 0 < node <
// n_nodes (node 0 is a root, never a child), so one unsigned compare of
// (v >> 11) - 1 with nn1 = n_nodes - 1 keeps every read in bounds; a walk
// that ends on a tag-0 entry other than the sentinel (a child out of range)
// is caught by walk_end_bad.  Returns whether an entry was read.
template <bool kRoot>
__device__ __forceinline__ uint32_t walk_step(const uint64_t* nodes, const uint64_t* root, const uint16_t* lut,
                                              Walk& w, uint64_t& v, uint32_t nn1) {
    const bool live = w.st == 1;
    const bool go = live && w.left > 0;
    const uint32_t byte = next_byte(lut, w);
    if (go) v = kRoot ? root[byte] : __ldg(nodes + (size_t)w.node * 256u + byte);
    const uint32_t lo = (uint32_t)v, child = (uint32_t)(v >> 11);
    const bool ptr = (lo & 3u) == 0u && child - 1u < nn1;
    if (go && ptr) w.node = child;
    if (live) w.st = go ? (ptr ? 1 : 0) : 2;
    return go ? 1u : 0u;
}

// A walk that ended (st 0) on a tag-0 entry other than the sentinel read a
// child pointer outside the node array.
__device__ __forceinline__ bool walk_end_bad(const Walk& w, uint64_t v) {
    return w.st == 0 && ((uint32_t)v & 3u) == 0u && v != 0ull;
}

// Walks of PPT points (w, after their face/prefix stage) advance level by
// level together, so their gathers (Listing "Probe Adaptive Cell Trie") are
// in flight at the same time.  After kLockLevels levels the walks still
// unfinished in the warp (tail: the warp's 32 PPT-entry shared buffer) are
// packed one per lane, so the deep levels of a few walks do not hold the
// whole warp for PPT slots each; their results come back through the same
// buffer.  Without a buffer the walks go on in step.  Points whose walk
// needs an uncertified key byte get their FP64 id and walk again alone
// (counted in *fallbacks); they reload their coordinates from pts[32 k]
// (the lane's points), so lat/lng need no registers during the walk.
// Returns the trie entries read.
template <int PPT>
__device__ __forceinline__ uint32_t walk_points(const DevIndex& X, const DevFace* faces, const uint16_t* lut,
                                                const uint64_t* s_root, Walk* w, const double2* pts, uint64_t e[PPT],
                                                uint64_t* err, uint32_t* fallbacks, uint4* tail) {
    uint32_t gathers = 0, bad = 0;
    const uint64_t* nodes = X.nodes;
    const uint32_t nn1 = (uint32_t)min(X.n_nodes, (uint64_t)0xFFFFFFFFu) - 1u;   // an index with walks has nodes
    uint64_t v[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) v[k] = 0;
    if (s_root) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) gathers += walk_step<true>(nodes, s_root, lut, w[k], v[k], nn1);
    } else {
#pragma unroll
        for (int k = 0; k < PPT; ++k) gathers += walk_step<false>(nodes, nullptr, lut, w[k], v[k], nn1);
    }
#pragma unroll
    for (int d = 1; d < kLockLevels; ++d) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) gathers += walk_step<false>(nodes, nullptr, lut, w[k], v[k], nn1);
    }
    uint32_t m[PPT], any = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        m[k] = __ballot_sync(kFull, w[k].st == 1);
        any |= m[k];
    }
    if (any) {
        if (tail) {
            const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
            uint32_t rank[PPT], n_tail = 0;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                rank[k] = n_tail + __popc(m[k] & lt);
                n_tail += __popc(m[k]);
                if (w[k].st == 1)
                    tail[rank[k]] = make_uint4(w[k].i32, w[k].j32, w[k].node, w[k].o | ((uint32_t)w[k].left << 11));
            }
            __syncwarp();
            for (uint32_t r0 = 0; r0 < n_tail; r0 += 32) {      // warp-uniform: one round unless > 32 walks
                const uint32_t r = r0 + lane;
                Walk x;
                x.st = 0;
                x.o = 0;
                x.i32 = x.j32 = x.node = 0;
                x.left = 0;
                uint64_t vx = 0;
                if (r < n_tail) {
                    const uint4 q = tail[r];
                    x.i32 = q.x;
                    x.j32 = q.y;
                    x.node = q.z;
                    x.o = q.w & 0x600u;
                    x.left = (int32_t)(q.w >> 11);
                    x.st = 1;
                }
                while (__any_sync(kFull, x.st == 1)) gathers += walk_step<false>(nodes, nullptr, lut, x, vx, nn1);
                if (walk_end_bad(x, vx)) bad = 1u;
                if (r < n_tail) tail[r] = make_uint4((uint32_t)vx, (uint32_t)(vx >> 32), (uint32_t)x.st, 0u);
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (w[k].st == 1) {
                    const uint4 q = tail[rank[k]];
                    v[k] = (uint64_t)q.x | ((uint64_t)q.y << 32);
                    w[k].st = (int32_t)q.z;
                }
            }
            __syncwarp();      // the buffer is free for the warp's next tile
        } else {
            // every walk ends within 8 key bytes (its certified bytes run out)
            bool more = true;
            for (int d = kLockLevels; d < 8 && more; ++d) {
                more = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    gathers += walk_step<false>(nodes, nullptr, lut, w[k], v[k], nn1);
                    more |= w[k].st == 1;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (walk_end_bad(w[k], v[k])) bad = 1u;
        e[k] = w[k].st == 0 ? v[k] : 0ull;
        if (w[k].st == 1) {
            bad = 1u;
        } else if (w[k].st == 2) {
            ++*fallbacks;
            Walk x;
            const double2 q = pts[32 * k];
            begin_walk(X, faces, lut, q.x, q.y, true, x);
            uint64_t vx = 0;
            while (x.st == 1) gathers += walk_step<false>(nodes, nullptr, lut, x, vx, nn1);
            // the FP64 id certifies every byte: a walk that uses them all up is corrupt
            if (x.st == 2 || walk_end_bad(x, vx)) bad = 1u;
            e[k] = x.st == 0 ? vx : 0ull;
        }
    }
    if (bad) atomicOr((unsigned long long*)err, (unsigned long long)kErrTrieBounds);
    return gathers;
}

// The probe of PPT points from their leaf cells (ok[k] false: point k is in
// no cell).
template <int PPT>
__device__ __forceinline__ uint32_t probe_cells(const DevIndex& X, const DevFace* faces, const uint16_t* lut,
                                                const uint64_t* s_root, const PointIJ* p, const bool* ok,
                                                const double2* pts, uint64_t e[PPT], uint64_t* err,
                                                uint32_t* fallbacks, uint4* tail) {
    Walk w[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        w[k].st = 0;
        w[k].o = 0;
        if (ok[k]) start_walk(faces, lut, p[k], w[k]);
    }
    return walk_points<PPT>(X, faces, lut, s_root, w, pts, e, err, fallbacks, tail);
}

// The probe of PPT points from their coordinates (valid[k] false: padding
// lane), cell id and face/prefix stage point by point.
template <int PPT>
__device__ __forceinline__ uint32_t probe_points(const DevIndex& X, const DevFace* faces, const uint16_t* lut,
                                                 const uint64_t* s_root, const double* lat, const double* lng,
                                                 const double2* pts, const bool* valid, uint64_t e[PPT],
                                                 uint64_t* err, uint32_t* fallbacks, uint4* tail) {
    Walk w[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        w[k].st = 0;
        w[k].o = 0;
        if (valid[k]) begin_walk(X, faces, lut, lat[k], lng[k], false, w[k]);
    }
    return walk_points<PPT>(X, faces, lut, s_root, w, pts, e, err, fallbacks, tail);
}

// Adds two per-thread counts (a < 2^15, b < 2^7 per thread) to two device
// counters with one warp reduction (a single redux instruction) and at most
// two atomics per warp.
__device__ __forceinline__ void warp_count2(uint32_t a, uint32_t b, uint64_t* ca, uint64_t* cb) {
    const uint32_t v = __reduce_add_sync(kFull, a | (b << 20));
    if ((threadIdx.x & 31) == 0) {
        if (v & 0xFFFFFu) atomicAdd((unsigned long long*)ca, (unsigned long long)(v & 0xFFFFFu));
        if (v >> 20) atomicAdd((unsigned long long*)cb, (unsigned long long)(v >> 20));
    }
}

// Adds a per-thread count to a device counter with one atomic per warp.
__device__ __forceinline__ void warp_count(uint32_t v, uint64_t* counter) {
    v = __reduce_add_sync(kFull, v);
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

// The first queue slot of each lane's candidates within its tile (lane-major,
// then point k: the lane's slots are the exclusive warp prefix of its
// candidate total csum) and the tile's total.  Nearly every candidate point
// has one candidate reference, so when no point of the warp has more, the
// prefix is a popcount of two ballots per point slot; otherwise a warp scan.
template <int PPT>
__device__ __forceinline__ uint32_t tile_slot_base(const uint32_t* nc, uint32_t csum, uint32_t* total) {
    bool multi = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) multi |= nc[k] > 1;
    if (__any_sync(kFull, multi)) {
        const uint32_t x = warp_incl_scan(csum);
        *total = __shfl_sync(kFull, x, 31);
        return x - csum;
    }
    const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
    uint32_t base = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint32_t m = __ballot_sync(kFull, nc[k] != 0);
        base += __popc(m & lt);
        tot += __popc(m);
    }
    *total = tot;
    return base;
}

// Per-CTA setup shared by the probe kernels: the Hilbert table in shared
// memory and, when every tile of the CTA probes the same index X (else
// null), its face table and, with the fast model, the model face's root
// node.  Returns the shared root (or null).
__device__ __forceinline__ const uint64_t* cta_setup(const DevIndex* X, uint16_t* s_hlut, DevFace* s_faces,
                                                     uint64_t* s_root) {
    for (int t = threadIdx.x; t < 512; t += blockDim.x)
        reinterpret_cast<uint32_t*>(s_hlut)[t] = reinterpret_cast<const uint32_t*>(g_hilbert_lut.v)[t];
    if (!X) return nullptr;
    if (threadIdx.x < 6) s_faces[threadIdx.x] = X->faces[threadIdx.x];
    if (!X->model.enabled) return nullptr;
    const uint32_t root = X->faces[X->model.face].root;
    if (root == kNoRootDev) return nullptr;
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(X->nodes + (uint64_t)root * 256);
    for (int t = threadIdx.x; t < 128; t += blockDim.x) reinterpret_cast<ulonglong2*>(s_root)[t] = __ldg(src + t);
    return s_root;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// A CTA's "tables ready" barrier (an mbarrier in shared memory, phase 0):
// every thread's cp.async copies arrive on it when they land (noinc: the
// expected count includes them), and the threads that store the face table
// arrive after their stores.  A warp that waits on it waits for the copies
// only, not for the CTA's other warps, as a CTA barrier would.
constexpr uint32_t kReadyArrivals = kJoinBlock + 6;
__device__ __forceinline__ void ready_init(uint64_t* bar, uint32_t arrivals = kReadyArrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(arrivals)
                 : "memory");
}
__device__ __forceinline__ void ready_arrive_on_copies(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}
__device__ __forceinline__ void ready_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}
__device__ __forceinline__ bool ready_test(uint32_t a) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(0u)
        : "memory");
    return done != 0;
}
// Waits (acquire) for phase 0 of the barrier: non-blocking tests, with a
// short sleep between them after the first, kSpinLimit of them at most
// (about a second, as the scan's look-back); false if it did not complete.
__device__ __forceinline__ bool ready_wait(uint64_t* bar) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    if (ready_test(a)) return true;
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        __nanosleep(32);
        if (ready_test(a)) return true;
    }
    return false;
}

// Bulk L2 prefetch of points p0 .. p0 + count - 1 (clipped to n; 16 bytes
// each, so the range is 16-byte aligned and a multiple of 16 bytes).
__device__ __forceinline__ void prefetch_points_l2(const double2* pts, uint64_t n, uint64_t p0, uint64_t count) {
    if (p0 >= n) return;
    const uint64_t c = min(count, n - p0);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pts + p0), "r"((uint32_t)(c * 16)) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// cta_setup for one index without the wait: the Hilbert table and the model
// face's root node go to shared memory as asynchronous 16-byte copies (one
// per thread of the 256), so the CTA computes its points' cell ids while
// they land; the face table is stored directly.  Every thread must call
// cp_async_wait_all and then __syncthreads before reading any of the three.
// Returns the shared root (or null).
// With ready (an initialised tables-ready barrier, see ready_init) the
// copies and the face stores arrive on it instead, and a warp reads the
// tables once ready_wait returns.
__device__ __forceinline__ const uint64_t* cta_setup_async(const DevIndex& X, uint16_t* s_hlut, DevFace* s_faces,
                                                           uint64_t* s_root, uint64_t* ready = nullptr) {
    static_assert(kJoinBlock == 256, "one 16-byte copy per thread: 128 for the table, 128 for the root");
    const uint32_t t = threadIdx.x;
    if (t < 128) cp_async16(s_hlut + 8 * t, g_hilbert_lut.v + 8 * t);
    const uint32_t root = X.model.enabled ? X.faces[X.model.face].root : kNoRootDev;
    if (root != kNoRootDev && t >= 128) cp_async16(s_root + 2 * (t - 128), X.nodes + (uint64_t)root * 256 + 2 * (t - 128));
    if (ready) ready_arrive_on_copies(ready);
    else cp_async_commit();
    if (t < 6) {
        s_faces[t] = X.faces[t];
        if (ready) ready_arrive(ready);
    }
    return root != kNoRootDev ? s_root : nullptr;
}

__device__ __forceinline__ uint32_t payload_of(uint64_t e, int which) {
    return (uint32_t)(e >> (which ? 33 : 2)) & 0x7FFFFFFFu;
}

// Writes every reference of entry e (approximate join), ascending ids.
__device__ __forceinline__ void emit_all(const DevIndex& X, uint64_t e, uint32_t* ids, uint64_t o) {
    const uint32_t tag = (uint32_t)(e & 3ull);
    if (tag == 1) {
        ids[o] = out_poly(X, payload_of(e, 0) >> 1);
    } else if (tag == 2) {
        ids[o] = out_poly(X, payload_of(e, 0) >> 1);
        ids[o + 1] = out_poly(X, payload_of(e, 1) >> 1);
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
            if (ta < cb) { ids[o++] = out_poly(X, ta); ++a; }
            else { ids[o++] = out_poly(X, cb); ++b; }
        }
    }
}


// ST_Covers in FP64 exactly as the spec (the certified test's fallback):
// same face, closed (u,v) bbox, ring rule with integer keys for the range
// tests and FP64 orientation, vertices read from global memory.  With
// X.contains (ST_Contains) a point on an edge or vertex is outside instead.
// The certified FP32 test never decides such a point (its orientation or a
// vertex lies within the error bounds), so this is the only place where the
// predicates differ.
__device__ __forceinline__ bool covers_fp64(const DevIndex& X, uint32_t poly, double lat, double lng) {
    if (!point_valid(lat, lng)) return false;
    double pu, pv;
    const int f = face_uv(lat, lng, &pu, &pv);
    if (f != X.poly_face[poly]) return false;
    const int64_t puk = dkey(pu), pvk = dkey(pv);
    const int64_t* bb = X.poly_bbox + 4ull * poly;
    if (!(puk >= bb[0] && puk <= bb[1] && pvk >= bb[2] && pvk <= bb[3])) return false;
    const uint32_t v0 = X.poly_off[poly], V = X.poly_off[poly + 1] - v0;
    const uint32_t r0 = X.ring_off[poly], r1 = X.ring_off[poly + 1];
    bool inside = false;
    for (uint32_t r = r0, start = 0;; ++r) {
        // edges (k, k + 1) for k in [start, stop): one ring -> every vertex
        // (the last edge wraps to vertex 0); with holes -> each ring up to
        // its closing copy of its first vertex
        const uint32_t stop = r1 > r0 ? X.ring_end[r] - 1 : V;
        for (uint32_t k = start; k < stop; ++k) {
            const uint32_t a = v0 + k, b = v0 + (k + 1 == V ? 0u : k + 1);
            const int64_t av = X.poly_vkey[a], bv = X.poly_vkey[b];
            const int64_t vlo = av < bv ? av : bv, vhi = av < bv ? bv : av;
            if (pvk < vlo || pvk > vhi) continue;
            const double2 A = X.poly_uv[a], B = X.poly_uv[b];
            const double o = (B.x - A.x) * (pv - A.y) - (B.y - A.y) * (pu - A.x);
            if (o == 0.0) {
                const int64_t au = X.poly_ukey[a], bu = X.poly_ukey[b];
                if (puk >= (au < bu ? au : bu) && puk <= (au < bu ? bu : au)) return X.contains == 0u;
            }
            if ((av <= pvk && pvk < bv && o > 0.0) || (bv <= pvk && pvk < av && o < 0.0)) inside = !inside;
        }
        if (r + 1 >= r1) break;
        start = X.ring_end[r];
    }
    return inside;
}

// ---------------------------------------------------------------------------
// job sources
// ---------------------------------------------------------------------------

// One (index, points, output) job.  Its warp tiles are tile0 .. tile0 +
// ceil(n / (32 PPT)) - 1 of the global tile space (in the batched form its
// range is padded to whole CTAs with tiles of no points), and in exact mode
// its index's polygons are poly0 .. poly0 + n_polys - 1 of the global
// polygon space of the refine step (shared by the jobs of one index).  Per-point work space (stored entries, queue bases) is
// indexed by the tile-padded global point index wt * 32 PPT + lane + 32 k,
// which needs no job lookup.
struct __align__(16) JobDesc {
    DevIndex X;
    const double2* pts;
    uint32_t* offsets;        // n + 1
    uint32_t* ids;
    uint64_t* status;         // 4 words: nnz, error bits, candidates, trie entries read
    uint64_t* counters;       // [0] FP64 cell-id fallbacks, [1] FP64 refine fallbacks
    uint64_t ids_cap;
    uint64_t tile0;
    uint32_t n;
    uint32_t poly0;
    uint32_t exact;           // 1: exact join (refine candidates), 0: approximate join
};

// The plain join: one job, passed by value as a kernel parameter.
struct OneJob {
    JobDesc d;
    static constexpr bool kSingle = true;
    __device__ __forceinline__ uint32_t find_tile(uint64_t) const { return 0; }
    __device__ __forceinline__ const JobDesc& job(uint32_t) const { return d; }
    __device__ __forceinline__ uint32_t job_base(uint32_t) const { return 0; }
};

// The batched form: m jobs in device memory, laid end to end, the
// approximate jobs' tiles first.  A probe or emit launch covers the tiles
// t0 .. T - 1 of one mode (t0 a multiple of the CTA's 8 tiles); ta is where
// the exact jobs' tiles begin.
struct ManyJobs {
    const JobDesc* d;
    const uint16_t* tile_job; // job of each global tile
    const uint32_t* base;     // per job: tile prefix (mod 2^32) at its first tile, written by the scan
    uint64_t t0;
    uint64_t ta;
    uint32_t m;
    static constexpr bool kSingle = false;
    __device__ __forceinline__ uint32_t find_tile(uint64_t wt) const { return __ldg(tile_job + wt); }
    __device__ __forceinline__ const JobDesc& job(uint32_t j) const { return d[j]; }
    __device__ __forceinline__ uint32_t job_base(uint32_t j) const { return base[j]; }
};

// Join mode of a kernel instance: fixed, or read from each job (batched form).
enum : int { kModeApprox = 0, kModeExact = 1, kModeAny = 2 };

template <int MODE>
__device__ __forceinline__ bool job_exact(const JobDesc& J) {
    return MODE == kModeAny ? J.exact != 0u : MODE == kModeExact;
}

// The work space of the join kernels (global tile and point spaces).
struct JoinScratch {
    uint64_t* entries;        // tagged trie entry per point
    uint32_t* tile_count;     // pairs per warp tile (exact: true hits, then + passing candidates)
    uint32_t* tile_prefix;    // exclusive scan of tile_count (mod 2^32)
    uint2* queue;             // exact: (global point, global polygon) candidates, tile_slots per tile
    uint8_t* pass;            // exact: PIP result per queue slot
    uint32_t* tile_cand;      // exact: candidates queued by each tile
    uint32_t* poly_count;     // exact: candidates per global polygon (k_count)
    uint32_t tile_slots;      // exact: queue slots per tile (32 PPT x most candidates of a point)
    const uint64_t* scan_err; // error bits of the scans, merged into each job's status
};

// ---------------------------------------------------------------------------
// join kernels
// ---------------------------------------------------------------------------

__global__ void k_zero(uint64_t* __restrict__ a, uint64_t na, uint64_t* __restrict__ b, uint64_t nb);

// Exact jobs: the tile's candidate references (nc[k] of point k, csum of
// the lane) go to the tile's own queue region, in point order (lane-major,
// then k), so no reservation is shared between tiles.
// The candidates queued are added to s_cnt[2] (a CTA's shared counter,
// flushed once per CTA) or, without one, to the job's status[2].
template <int PPT>
__device__ __forceinline__ void queue_tile(const JobDesc& J, const uint64_t* e, const uint32_t* nc, uint32_t csum,
                                           uint64_t wt, uint64_t gbase, uint32_t gpoly0, const JoinScratch& S,
                                           uint32_t* s_cnt = nullptr) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t wtotal;
    const uint32_t first = tile_slot_base<PPT>(nc, csum, &wtotal);
    if (lane == 0) {
        S.tile_cand[wt] = wtotal;
        if (wtotal) {
            if (s_cnt) atomicAdd(&s_cnt[2], wtotal);
            else atomicAdd((unsigned long long*)&J.status[2], (unsigned long long)wtotal);
        }
    }
    if (wtotal == 0) return;
    if (wtotal > S.tile_slots) {    // cannot happen: a point has at most the index's candidate references
        if (lane == 0) atomicOr((unsigned long long*)&J.status[1], (unsigned long long)kErrQueueOverflow);
        return;
    }
    uint2* q = S.queue + wt * S.tile_slots + first;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint32_t g = (uint32_t)(gbase + lane + 32 * k);     // global point index
        const uint64_t ek = e[k];
        const uint32_t tag = (uint32_t)(ek & 3ull);
        if (tag != 3) {
            // inline references (nearly every candidate): candidate = interior bit clear
            const uint32_t p0 = payload_of(ek, 0), p1 = payload_of(ek, 1);
            const bool c0 = nc[k] != 0 && (p0 & 1u) == 0u;
            const bool c1 = tag == 2 && (p1 & 1u) == 0u;
            if (c0) *q = make_uint2(g, gpoly0 + (p0 >> 1));
            if (c1) q[c0 ? 1 : 0] = make_uint2(g, gpoly0 + (p1 >> 1));
            q += nc[k];
        } else if (nc[k]) {
            const uint32_t off = payload_of(ek, 0);
            const uint32_t* Cc = J.X.lut + off + 2 + __ldg(J.X.lut + off);
            for (uint32_t r = 0; r < nc[k]; ++r) q[r] = make_uint2(g, gpoly0 + __ldg(Cc + r));
            q += nc[k];
        }
    }
}

// Step 1 of the join (Listing "Probe Adaptive Cell Trie" per point) for
// warp tile wt = tile lt of job J: cell id + walk for every point of the tile (32 lanes x PPT
// points, point base + lane + 32 k, so the 16-byte loads coalesce), the
// tagged entry stored per point.  Approximate jobs count every reference of
// the tile; exact jobs count the true hits and write the candidate
// references to the tile's own queue region (queue_tile).  No tile waits on
// another.
// With kAsync the CTA's shared tables are still in flight (cta_setup_async):
// every thread of the CTA calls this (active false: a warp past the last
// tile), and the wait comes after the cell ids, before the first table
// read: on the tables-ready barrier `ready` when given, else a copy wait and
// a CTA barrier.  With `loaded` the caller loaded the tile's points
// (load_tile_points) before the CTA's setup.
// With s_cnt (a CTA's shared counters: trie entries read, FP64 fallbacks,
// candidates queued; zeroed before the CTA's barrier) the tile adds its
// counts there and the kernel flushes them once per CTA (flush_cta_counts):
// per-tile global atomics on the job's status words all hit one 32-byte
// sector and serialise in its L2 slice.  Without it they go to the job's
// status words directly.
// Loads the points of tile lt of job J (lane + 32 k) into q; lanes past
// the job's last point (or an inactive warp) get zeros, which the tile
// does not use.
template <int PPT>
__device__ __forceinline__ void load_tile_points(const JobDesc& J, uint64_t lt, bool active, double2* q) {
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = lt * (32 * PPT) + (threadIdx.x & 31) + 32 * k;
        q[k] = make_double2(0.0, 0.0);
        if (active && p < J.n) q[k] = __ldcs(J.pts + p);      // streamed once
    }
}

// The start of a probe CTA: zeroes its n_cnt shared counters and (with
// AGJ_PROBE_READY_BARRIER) initialises its tables-ready barrier, then the
// CTA's one barrier makes both visible.  Returns the barrier (or null: the
// tile waits on a CTA barrier after its cell ids instead).
__device__ __forceinline__ uint64_t* cta_begin(uint32_t* s_cnt, int n_cnt, uint64_t* s_ready) {
    if ((int)threadIdx.x < n_cnt) s_cnt[threadIdx.x] = 0;
    if (!AGJ_PROBE_READY_BARRIER) return nullptr;
    if (threadIdx.x == 0) ready_init(s_ready);
    __syncthreads();
    return s_ready;
}

// Should the wait on `ready` ever give up, the tile joins nothing and sets
// the timed-out-wait bit of status[1].
template <int PPT, int MODE, bool kAsync = false>
__device__ __forceinline__ void probe_tile(const JobDesc& J, const DevFace* faces, const uint16_t* s_hlut,
                                           const uint64_t* s_root, uint64_t wt, uint64_t lt, uint32_t gpoly0,
                                           const JoinScratch& S, bool active = true, uint32_t* s_cnt = nullptr,
                                           uint4* tail = nullptr, uint64_t* ready = nullptr,
                                           const double2* loaded = nullptr) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t base = lt * (32 * PPT);
    const uint64_t gbase = wt * (32 * PPT);
    uint64_t e[PPT];
    uint32_t fallbacks = 0;
    PointIJ pij[PPT];
    bool ok[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        ok[k] = false;
        if (active && p < J.n) {
            const double2 q = loaded ? loaded[k] : __ldcs(J.pts + p);     // streamed once
            ok[k] = point_ij(J.X.model, q.x, q.y, false, pij[k]);
        }
    }
    if constexpr (kAsync) {
        if (ready) {
            if (!active) return;
            if (!ready_wait(ready)) {
                // the tile's points join nothing and no walk reads the
                // tables; the join reports the timed-out wait
                if (lane == 0) atomicOr((unsigned long long*)&J.status[1], (unsigned long long)kErrScanTimeout);
#pragma unroll
                for (int k = 0; k < PPT; ++k) ok[k] = false;
            }
        } else {
            cp_async_wait_all();
            __syncthreads();
        }
    }
    if (!active) return;
    const uint32_t gathers = probe_cells<PPT>(J.X, faces, s_hlut, s_root, pij, ok, J.pts + base + lane, e,
                                              &J.status[1], &fallbacks, tail);
    if (s_cnt) {
        const uint32_t g = __reduce_add_sync(kFull, gathers), f = __reduce_add_sync(kFull, fallbacks);
        if (lane == 0) {
            if (g) atomicAdd(&s_cnt[0], g);
            if (f) atomicAdd(&s_cnt[1], f);
        }
    } else {
        warp_count2(gathers, fallbacks, &J.status[3], &J.counters[0]);
    }
    const bool exact = job_exact<MODE>(J);
    uint32_t nc[PPT], csum = 0, tsum = 0;    // nc: candidates the point queues (none for approximate jobs)
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        uint32_t nt, n_cand;
        entry_counts(J.X, e[k], &nt, &n_cand);
        tsum += exact ? nt : nt + n_cand;
        nc[k] = exact ? n_cand : 0u;
        csum += nc[k];
        S.entries[gbase + lane + 32 * k] = e[k];        // 0 for padding lanes
    }
    tsum = __reduce_add_sync(kFull, tsum);
    if (lane == 0) S.tile_count[wt] = tsum;
    if constexpr (MODE != kModeApprox) {
        if (S.tile_cand) queue_tile<PPT>(J, e, nc, csum, wt, gbase, gpoly0, S, s_cnt);
    } else {
        if (S.tile_cand && lane == 0) S.tile_cand[wt] = 0;      // a batched plan's approximate tile
    }
}

// Adds a CTA's shared counters (see probe_tile) to job J's status words
// and diagnostics; called by every thread after the CTA's tiles.
__device__ __forceinline__ void flush_cta_counts(const JobDesc& J, const uint32_t* s_cnt) {
    asm volatile("cp.async.wait_all;" ::: "memory");   // no copy of the CTA's outlives it
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt[0]) atomicAdd((unsigned long long*)&J.status[3], (unsigned long long)s_cnt[0]);
        if (s_cnt[1]) atomicAdd((unsigned long long*)&J.counters[0], (unsigned long long)s_cnt[1]);
        if (s_cnt[2]) atomicAdd((unsigned long long*)&J.status[2], (unsigned long long)s_cnt[2]);
    }
}

// Stages job J's face table and (with the fast model) the model face's root
// node in shared memory.  Called by the whole CTA for a CTA-uniform job.
// (The descriptor itself stays in global memory: read through the cache, its
// fields are reloaded where needed instead of being held in registers.)
__device__ __forceinline__ const uint64_t* cta_stage_job(const JobDesc& J, DevFace* s_faces, uint64_t* s_root) {
    __syncthreads();   // the previous job's tiles are done with the staged copy
    const DevIndex& X = J.X;
    if (threadIdx.x < 6) s_faces[threadIdx.x] = X.faces[threadIdx.x];
    const uint64_t* root = nullptr;
    if (X.model.enabled && X.faces[X.model.face].root != kNoRootDev) {
        const ulonglong2* r = reinterpret_cast<const ulonglong2*>(X.nodes + (uint64_t)X.faces[X.model.face].root * 256);
        for (int t = threadIdx.x; t < 128; t += blockDim.x) reinterpret_cast<ulonglong2*>(s_root)[t] = __ldg(r + t);
        root = s_root;
    }
    __syncthreads();
    return root;
}

// The plain join runs one warp per tile of its single job (job offsets are
// compile-time zero).  The batched form aligns every job's tile range to
// whole CTAs, so the 8 tiles a CTA takes at a time belong to one job, whose
// face table and root node the CTA stages in shared memory when the job
// changes; the grid either covers the tile space (one warp per tile) or, with
// kPersist, is persistent and strides over it (separate instances, so the
// one-warp-per-tile form carries no loop state).
// Resident CTAs per SM a probe instance is compiled for.
template <int PPT, class Src, int MODE>
constexpr int probe_min_blocks() {
    return MODE == kModeApprox ? (Src::kSingle && PPT >= 4 ? AGJ_JOIN_APPROX_PROBE_MIN_BLOCKS : AGJ_APPROX_PROBE_MIN_BLOCKS)
           : !Src::kSingle     ? AGJ_BATCH_PROBE_MIN_BLOCKS
                               : AGJ_PROBE_MIN_BLOCKS;
}

template <int PPT, class Src, int MODE, bool kPersist = false>
__global__ void __launch_bounds__(kJoinBlock, probe_min_blocks<PPT, Src, MODE>())
    k_probe(const Src src, uint64_t T, const JoinScratch S) {
    __shared__ __align__(16) uint16_t s_hlut[1024];
    __shared__ __align__(16) uint64_t s_rootbuf[256];
    __shared__ DevFace s_faces[6];
    __shared__ uint32_t s_cnt[3];
    __shared__ uint4 s_tail[kWarpsPerBlock][32 * PPT];
    __shared__ uint64_t s_ready;
    const uint32_t warp = threadIdx.x >> 5;
    if constexpr (Src::kSingle) {
        // the tile's point loads are issued first; then the tables-ready
        // barrier and the shared counters are set up before the CTA's one
        // barrier ahead of the tile, and each warp waits for the table
        // copies alone (its cell ids overlap them)
        const uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;
        double2 q[PPT];
        if (AGJ_PROBE_READY_BARRIER) load_tile_points<PPT>(src.job(0), wt, wt < T, q);
        uint64_t* ready = cta_begin(s_cnt, 3, &s_ready);
        const uint64_t* s_root = cta_setup_async(src.job(0).X, s_hlut, s_faces, s_rootbuf, ready);
        if (threadIdx.x == 32) {
            // the points of the CTA one full grid of resident CTAs ahead go
            // to the L2 now, so that CTA finds them there
            uint32_t nsm;
            asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
            const uint64_t group_pts = (uint64_t)kWarpsPerBlock * 32 * PPT;
            const uint64_t ahead = (uint64_t)nsm * probe_min_blocks<PPT, Src, MODE>();
            if (AGJ_PREFETCH_AHEAD) prefetch_points_l2(src.job(0).pts, src.job(0).n, (blockIdx.x + ahead) * group_pts, group_pts);
        }
        probe_tile<PPT, MODE, true>(src.job(0), s_faces, s_hlut, s_root, wt, wt, 0, S, wt < T, s_cnt, s_tail[warp],
                                    ready, AGJ_PROBE_READY_BARRIER ? q : nullptr);
        flush_cta_counts(src.job(0), s_cnt);
    } else {
        const uint64_t g0 = src.t0 / kWarpsPerBlock;
        if constexpr (!kPersist) {                                  // one CTA per 8 tiles of one job
            const uint64_t g = g0 + blockIdx.x;
            if (g * kWarpsPerBlock >= T) return;
            const JobDesc& J = src.job(src.find_tile(g * kWarpsPerBlock));
            const uint64_t wt = g * kWarpsPerBlock + warp;
            double2 q[PPT];
            if (AGJ_PROBE_READY_BARRIER) load_tile_points<PPT>(J, wt - J.tile0, true, q);
            uint64_t* ready = cta_begin(s_cnt, 3, &s_ready);
            const uint64_t* s_root = cta_setup_async(J.X, s_hlut, s_faces, s_rootbuf, ready);
            probe_tile<PPT, MODE, true>(J, s_faces, s_hlut, s_root, wt, wt - J.tile0, J.poly0, S, true, s_cnt,
                                        s_tail[warp], ready, AGJ_PROBE_READY_BARRIER ? q : nullptr);
            flush_cta_counts(J, s_cnt);
        } else {                                                    // persistent grid
            cta_setup(nullptr, s_hlut, s_faces, s_rootbuf);
            uint32_t cur = 0xFFFFFFFFu;
            const uint64_t* s_root = nullptr;
            for (uint64_t g = g0 + blockIdx.x; g * kWarpsPerBlock < T; g += gridDim.x) {
                const uint32_t j = src.find_tile(g * kWarpsPerBlock);
                const JobDesc& J = src.job(j);
                if (j != cur) {
                    s_root = cta_stage_job(J, s_faces, s_rootbuf);
                    cur = j;
                }
                const uint64_t wt = g * kWarpsPerBlock + warp;
                probe_tile<PPT, MODE>(J, s_faces, s_hlut, s_root, wt, wt - J.tile0, J.poly0, S, true, nullptr,
                                      s_tail[warp]);
            }
        }
    }
}

// Exclusive scan of the tile counts over the whole tile space: CTA chunks of
// 16 x 256 counts chained by the decoupled look-back (a few hundred chunks,
// so the look-back is short).  Prefixes are kept mod 2^32: a job's offsets are
// differences of two prefixes of its own tiles.
// With tile_job (batched form), the prefix at each job's first tile is also
// written to job_base[job].
__global__ void k_scan_counts(const uint32_t* __restrict__ tile_count, uint64_t m, uint32_t* __restrict__ tile_prefix,
                              uint64_t* __restrict__ chunks, uint32_t* __restrict__ chunk_counter,
                              uint64_t* __restrict__ err, const uint16_t* __restrict__ tile_job,
                              uint32_t* __restrict__ job_base);

// Exclusive scans of the per-polygon candidate counts and of the per-polygon
// refine chunks (kPipBlock candidates each), as one packed 64-bit scan
// (count in the low 32 bits, chunks above) chained by the look-back; each
// refine chunk's (polygon, first candidate, candidates) goes to chunk_desc.
// The CTA that finishes last writes the refine chunk count; cursor receives
// each polygon's first slot in the grouped order (the scatter's cursors).
__global__ void k_poly_scan(const uint32_t* __restrict__ poly_count, uint32_t n_polys,
                            uint32_t* __restrict__ cursor, uint32_t* __restrict__ n_chunks,
                            uint4* __restrict__ chunk_desc, uint64_t* __restrict__ chunks,
                            uint32_t* __restrict__ chunk_counter, uint64_t* __restrict__ err);

// Candidates per polygon of the queue (tile_cand[t] items from slot
// t x tile_slots of each tile t), taken in chunks of chunk_tiles tiles
// (a power of two, 32 .. 512).
__global__ void k_count(const uint2* __restrict__ queue, const uint32_t* __restrict__ tile_cand, uint64_t n_tiles,
                        uint32_t tile_slots, uint32_t chunk_tiles, uint32_t* __restrict__ poly_count,
                        uint32_t n_polys);

// Groups the queued candidates by polygon: a counting-sort scatter of
// (global point, queue slot) pairs, same chunks as k_count.
__global__ void k_scatter(const uint2* __restrict__ queue, const uint32_t* __restrict__ tile_cand, uint64_t n_tiles,
                          uint32_t tile_slots, uint32_t chunk_tiles, uint32_t* __restrict__ cursor,
                          uint2* __restrict__ sorted, uint32_t n_polys);

// Tiles per chunk of k_count / k_scatter: 512 for large queues, smaller ones
// split so that about four chunks per SM share the work, but at least
// n_polys / 8 tiles, since k_scatter clears and reserves its shared
// counters (one per polygon) once per chunk.
inline uint32_t refine_chunk_tiles(uint64_t n_tiles, int sms, uint64_t n_polys) {
    uint32_t ct = 32;
    while (ct < 512 && ((uint64_t)ct * 4 * (uint64_t)sms < n_tiles || (uint64_t)ct * 8 < n_polys)) ct <<= 1;
    return ct;
}

// Grids of the candidate grouping (k_count, k_scatter): both stride over
// chunks of ct tiles; per_sm CTAs per SM at most, and no more CTAs than
// chunks.  Their work per item is a short chain of dependent loads and a
// shared atomic, so they want many warps in flight: 6 CTAs per SM (as many
// as their 34 KB of shared memory each allow) against 2 and 4 took the
// city refine from 0.56 to 0.50 ms per 1e8 points (4 and 4: 0.52 ms).
#ifndef AGJ_COUNT_CTAS_PER_SM
#define AGJ_COUNT_CTAS_PER_SM 6
#endif
#ifndef AGJ_SCATTER_CTAS_PER_SM
#define AGJ_SCATTER_CTAS_PER_SM 6
#endif
inline int refine_sort_grid(uint64_t n_tiles, uint32_t ct, int sms, int per_sm) {
    const uint64_t chunks = (n_tiles + ct - 1) / ct;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(chunks, (uint64_t)sms * per_sm));
}

// Refine (Listing "Join" step 3 on candidate references): ST_Covers of
// (point, polygon) candidates, grouped by polygon.  Per chunk of one
// polygon's candidates, the polygon's FP32 local vertices are staged in
// shared memory and every thread tests its candidate against the same edge at
// the same time (shared-memory broadcast).  The test is the certified FP32
// one (covers_certified); an undecided candidate (within the error bounds of
// a vertex or an edge) is recomputed in FP64 (covers_fp64), as is every
// candidate of a polygon too large for the FP32 local frame.  A passing
// candidate adds one to its tile's pair count.  The polygon's data comes
// from the job of the chunk's first candidate (every job sharing a polygon
// range probes the same index); each candidate's point from its own job.
#ifndef AGJ_PIP_MIN_BLOCKS
#define AGJ_PIP_MIN_BLOCKS 6
#endif
//
// With kCount (aggregation mode) the candidates' results are not stored:
// the chunk's passing candidates (all of one polygon) are counted with one
// block reduction and added to counts[polygon] and to the pair count
// status[0] of the chunk's job.
constexpr int kPipSmemBand = 4096;               // band-table words staged per CTA (uint16)
template <class Src, bool kCount = false>
__global__ void __launch_bounds__(kPipBlock, AGJ_PIP_MIN_BLOCKS) k_pip(const Src src, uint32_t tile_points,
                                                                   const uint2* __restrict__ sorted,
                                                                   const uint4* __restrict__ chunk_desc,
                                                                   const uint32_t* __restrict__ n_chunks,
                                                                   uint8_t* __restrict__ pass,
                                                                   uint32_t* __restrict__ tile_count,
                                                                   uint64_t* __restrict__ counts = nullptr) {
    __shared__ F2 s_lv[kPipSmemVerts];
    __shared__ uint16_t s_band[kPipSmemBand];
    const uint32_t total = *n_chunks;
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        const uint4 cd = chunk_desc[c];                   // (polygon, first candidate, candidates)
        const uint32_t gp = cd.x;
        const bool have = threadIdx.x < cd.z;
        // the candidate and its point do not depend on the polygon's data:
        // their loads overlap the staging below
        uint2 it = make_uint2(0u, 0u);
        double2 pt = make_double2(0.0, 0.0);
        if (have) {
            it = sorted[cd.y + threadIdx.x];              // (global point, queue slot)
            const JobDesc& J = src.job(src.find_tile(it.x / tile_points));
            pt = J.pts[it.x - J.tile0 * tile_points];
        }
        const JobDesc& JP = src.job(src.find_tile(sorted[cd.y].x / tile_points));
        const uint32_t poly = gp - JP.poly0;
        const uint32_t v0 = JP.X.poly_off[poly], V = JP.X.poly_off[poly + 1] - v0;
        const PolyLocal L = JP.X.poly_local[poly];
        const bool certified = JP.X.model.uv_enabled && L.ok && V <= (uint32_t)kPipSmemVerts;
        const bool banded = certified && L.nb && L.band_len <= (uint32_t)kPipSmemBand;
        __syncthreads();
        if (certified)
            for (uint32_t t = threadIdx.x; t < V; t += blockDim.x) s_lv[t] = JP.X.poly_luv[v0 + t];
        if (banded)
            for (uint32_t t = threadIdx.x; t < L.band_len; t += blockDim.x) s_band[t] = JP.X.poly_band[L.band + t];
        __syncthreads();
        int r = 0;
        if (have) {
            const uint32_t wt = it.x / tile_points;
            r = -1;
            float pu, pv, dp;
            if (certified && model_uv_local(JP.X.model, pt.x, pt.y, L, &pu, &pv, &dp))
                r = covers_certified(s_lv, V, L, banded ? s_band : nullptr, pu, pv, dp);
            if (r < 0) {
                r = covers_fp64(JP.X, poly, pt.x, pt.y) ? 1 : 0;
                atomicAdd((unsigned long long*)&src.job(src.find_tile(wt)).counters[1], 1ull);
            }
            if constexpr (!kCount) {
                pass[it.y] = (uint8_t)r;
                if (r) atomicAdd(&tile_count[wt], 1u);
            }
        }
        if constexpr (kCount) {
            const int passed = __syncthreads_count(r);
            if (threadIdx.x == 0 && passed) {
                atomicAdd((unsigned long long*)&counts[out_poly(JP.X, poly)], (unsigned long long)passed);
                atomicAdd((unsigned long long*)&JP.status[0], (unsigned long long)passed);
            }
        }
    }
}

// Last step of the join (Listing "Join", add to pairs) for warp tile wt =
// tile lt of job j: offsets and ids of the tile from its stored entries and
// its prefix (less the prefix at the job's first tile), ids ascending
// per point (true and candidate references merged; exact jobs keep the
// candidates that passed).  The job's last tile writes offsets[n] and nnz.
template <int PPT, int MODE, class Src>
__device__ __forceinline__ void emit_tile(const Src& src, uint32_t j, uint64_t wt, const JoinScratch& S,
                                          uint8_t* s_pass) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gbase = wt * (32 * PPT);
    // the stored entries and the tile prefix do not depend on the job, so
    // their loads overlap the job lookup
    uint64_t e[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) e[k] = __ldcs(S.entries + gbase + lane + 32 * k);
    const uint32_t tprefix = S.tile_prefix[wt];
    const JobDesc& J = src.job(j);
    const bool exact = job_exact<MODE>(J);
    // exact: the first 32 PIP results of the tile's queue region, one per
    // lane, loaded beside the entries (the region's size is known only
    // after them)
    const uint32_t pb0 = (MODE != kModeApprox && exact) ? S.pass[wt * S.tile_slots + lane] : 0u;
    const uint64_t base = (wt - J.tile0) * (32 * PPT);
    uint32_t cnt[PPT], pm[PPT], qb[PPT], ex[PPT], run = 0;   // pm: bit t = candidate t of the point passed
    bool direct = false;     // a point with more than 32 candidates: read its results from memory
    if (exact) {
        // the queue slots of this tile's candidates, in the order the probe
        // wrote them: lane-major, then k
        uint32_t nt[PPT], nc[PPT], csum = 0, mx = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            entry_counts(J.X, e[k], &nt[k], &nc[k]);
            csum += nc[k];
            mx = nc[k] > mx ? nc[k] : mx;
            pm[k] = 0;
        }
        uint32_t unused_total;
        const uint32_t q0 = tile_slot_base<PPT>(nc, csum, &unused_total);
        mx = __reduce_max_sync(kFull, mx);
        direct = mx > 32;
        uint32_t qq = q0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            qb[k] = qq;
            qq += nc[k];
        }
        // the tile's first 32 results through the warp's shared bytes; the
        // rest (rare) from memory
        __syncwarp();                  // the warp's previous tile is done with its bytes
        s_pass[threadIdx.x] = (uint8_t)pb0;
        __syncwarp();
        const uint8_t* sp = s_pass + (threadIdx.x & ~31u);
        const uint8_t* gp = S.pass + wt * S.tile_slots;
        if (!direct) {
            // inline entries queue at most two candidates: their two result
            // bytes unrolled; longer lists (lookup-table cells) in a loop
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
#pragma unroll
                for (uint32_t t = 0; t < 2; ++t) {
                    const uint32_t idx = qb[k] + t;
                    if (t < nc[k] && (idx < 32 ? sp[idx] : gp[idx])) pm[k] |= 1u << t;
                }
                for (uint32_t t = 2; t < nc[k]; ++t) {
                    const uint32_t idx = qb[k] + t;
                    if (idx < 32 ? sp[idx] : gp[idx]) pm[k] |= 1u << t;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (!direct) {
                cnt[k] = nt[k] + __popc(pm[k]);
            } else {
                cnt[k] = nt[k];
                for (uint32_t t = 0; t < nc[k]; ++t) cnt[k] += S.pass[wt * S.tile_slots + qb[k] + t];
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            uint32_t nt, nc;
            entry_counts(J.X, e[k], &nt, &nc);
            cnt[k] = nt + nc;
            pm[k] = 0;
            qb[k] = 0;
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint32_t incl = warp_incl_scan(cnt[k]);
        ex[k] = run + incl - cnt[k];
        run += __shfl_sync(kFull, incl, 31);
    }
    const uint64_t prefix = (uint64_t)(uint32_t)(tprefix - src.job_base(j));
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const uint64_t p = base + lane + 32 * k;
        if (p >= J.n) continue;
        const uint64_t o = prefix + ex[k];
        __stcs(J.offsets + p, (uint32_t)o);
        if (!cnt[k]) continue;
        if (o + cnt[k] > J.ids_cap) {
            atomicOr((unsigned long long*)&J.status[1], (unsigned long long)kErrIdsCapacity);
            continue;
        }
        if (!exact) {
            emit_all(J.X, e[k], J.ids, o);
            continue;
        }
        const uint64_t ek = e[k];
        const uint32_t tag = (uint32_t)(ek & 3ull);
        const uint32_t ps = pm[k];
        const uint8_t* pd = S.pass + wt * S.tile_slots + qb[k];     // the results themselves (direct)
        uint64_t w = o;
        uint32_t ci = 0;
        if ((tag == 1 || tag == 2) && !direct) {
            // a true reference is kept, a candidate when its result bit is
            // set (bit 0 for the first candidate, bit 1 for a second)
            const uint32_t p0 = payload_of(ek, 0), p1 = payload_of(ek, 1);
            const bool keep0 = (p0 & 1u) || (ps & 1u);
            const bool keep1 = tag == 2 && ((p1 & 1u) || ((ps >> ((p0 & 1u) ? 0 : 1)) & 1u));
            if (keep0) J.ids[w] = out_poly(J.X, p0 >> 1);
            if (keep1) J.ids[w + (keep0 ? 1 : 0)] = out_poly(J.X, p1 >> 1);
        } else if (tag == 1 || tag == 2) {
            for (int t = 0; t < (int)tag; ++t) {
                const uint32_t pl = payload_of(ek, t);
                if (pl & 1u) J.ids[w++] = out_poly(J.X, pl >> 1);
                else if (pd[ci++]) J.ids[w++] = out_poly(J.X, pl >> 1);
            }
        } else if (tag == 3) {
            const uint32_t off = payload_of(ek, 0);
            const uint32_t nt = __ldg(J.X.lut + off);
            const uint32_t* Tt = J.X.lut + off + 1;
            const uint32_t nc = __ldg(J.X.lut + off + 1 + nt);
            const uint32_t* Cc = J.X.lut + off + 2 + nt;
            uint32_t a = 0, b = 0;
            while (a < nt || b < nc) {
                const uint32_t ta = a < nt ? __ldg(Tt + a) : 0xFFFFFFFFu;
                const uint32_t cb = b < nc ? __ldg(Cc + b) : 0xFFFFFFFFu;
                if (ta < cb) { J.ids[w++] = out_poly(J.X, ta); ++a; }
                else { if (direct ? pd[b] : (ps >> b) & 1u) J.ids[w++] = out_poly(J.X, cb); ++b; }
            }
        }
    }
    if (base < J.n && base + 32 * PPT >= J.n && lane == 0) {     // the job's last point

        J.offsets[J.n] = (uint32_t)(prefix + run);
        J.status[0] = prefix + run;
        const uint64_t g = *S.scan_err;
        if (g) atomicOr((unsigned long long*)&J.status[1], (unsigned long long)g);
    }
}

template <int PPT, class Src, int MODE>
__global__ void __launch_bounds__(kJoinBlock) k_emit(const Src src, uint64_t T, const JoinScratch S) {
    __shared__ uint8_t s_pass[kJoinBlock];
    uint64_t wt = (uint64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if constexpr (Src::kSingle) {
        if (wt < T) emit_tile<PPT, MODE>(src, 0, wt, S, s_pass);
    } else {
        wt += src.t0;
        if ((uint64_t)gridDim.x * kWarpsPerBlock >= T - src.t0) {   // one warp per tile
            if (wt < T) emit_tile<PPT, MODE>(src, src.find_tile(wt), wt, S, s_pass);
        } else {                                                     // persistent grid
            for (; wt < T; wt += (uint64_t)gridDim.x * kWarpsPerBlock)
                emit_tile<PPT, MODE>(src, src.find_tile(wt), wt, S, s_pass);
        }
    }
}

}  // namespace agj
