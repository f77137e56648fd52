// agj_device.cuh — device-side view of an index and the per-point probe
// steps (cell id, face/prefix stage, trie walk, entry decode).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "agj_geom.cuh"

namespace agj {

struct DevFace {
    uint32_t root;          // node index, 0xFFFFFFFF = no cells on this face
    uint32_t prefix_bits;   // key bits after the face bits (multiple of 8)
    uint64_t prefix;        // right-aligned
    // The prefix as a cell: a leaf (i, j) lies in it iff ((i ^ pi) | (j ^ pj))
    // & pmask == 0 (pi, pj: the cell's coordinates at level prefix_bits / 2,
    // shifted up to level 30); o_row: the Hilbert orientation after the
    // prefix levels, times 512 (the byte offset of its row in the walk's
    // lookup table of 2-byte entries).
    uint32_t pi, pj, pmask, o_row;
};

// Everything a kernel needs from one index; passed by value.
struct DevIndex {
    const uint64_t* nodes;      // n_nodes x 256 tagged entries
    const uint32_t* lut;        // lookup table
    const double2* poly_uv;     // polygon vertices in face (u,v)
    const int64_t* poly_vkey;   // order-preserving integer keys of the vertices' v
    const int64_t* poly_ukey;   // ... and of u
    const uint32_t* poly_off;   // n_polys + 1
    const int64_t* poly_bbox;   // 4 keys per polygon: umin umax vmin vmax
    const int8_t* poly_face;
    const PolyLocal* poly_local;  // certified refine: per-polygon reference, bound, bbox
    const F2* poly_luv;           // certified refine: FP32 local vertex coordinates
    const uint16_t* poly_band;    // certified refine: per-polygon band tables
    const uint32_t* ring_off;     // n_polys + 1: each polygon's entries in ring_end (none: one ring)
    const uint32_t* ring_end;     // ends of a polygon with holes' rings (explicitly closed), relative to poly_off
    const uint32_t* piece_poly;   // input polygon of each piece (null: piece k = polygon k)
    uint64_t n_nodes;
    uint64_t n_lut;
    uint32_t n_polys;           // pieces (the polygons of the references and the refine)
    uint32_t n_out_polys;       // input polygons (the ids of joins and counts)
    uint32_t max_depth;
    uint32_t contains;          // 1: the refine test excludes the boundary (ST_Contains)
    DevFace faces[6];
    FastModel model;            // certified fast cell ids (enabled == 0: FP64 ids)
};

constexpr uint32_t kNoRootDev = 0xFFFFFFFFu;
constexpr uint32_t kInvalidPayloadDev = 0x7FFFFFFFu;

// Error flag bits in status[1].
constexpr uint64_t kErrIdsCapacity = 1ull << 0;
constexpr uint64_t kErrScanTimeout = 1ull << 1;
constexpr uint64_t kErrTrieBounds = 1ull << 2;
constexpr uint64_t kErrQueueOverflow = 1ull << 3;

// Order-preserving map of a double onto int64 (sign-magnitude to two's
// complement); -0.0 and +0.0 map to the same key, so comparisons of keys
// equal IEEE comparisons for non-NaN values.
AGJ_HD int64_t dkey(double x) {
#ifdef __CUDA_ARCH__
    const int64_t b = __double_as_longlong(x);
#else
    int64_t b;
    memcpy(&b, &x, 8);
#endif
    return b < 0 ? -(b & 0x7FFFFFFFFFFFFFFFll) : b;
}

// Walks the trie for one leaf cell id computed by the FP64 spec (Listing
// "Probe Adaptive Cell Trie"): face bits select the root, the root's common
// prefix must match, then one key byte per level until the entry is not a
// child pointer.  Returns the final tagged entry (0 = false hit).
__device__ __forceinline__ uint64_t walk_exact(const DevIndex& X, const DevFace* faces, uint64_t id, uint64_t* err,
                                               uint32_t* gathers) {
    if (id == kInvalidId) return 0;
    const DevFace fr = faces[id >> 61];
    if (fr.root == kNoRootDev) return 0;
    uint64_t key = id << 3;
    if (fr.prefix_bits) {
        if ((key >> (64 - fr.prefix_bits)) != fr.prefix) return 0;
        key <<= fr.prefix_bits;
    }
    const char* base = reinterpret_cast<const char*>(X.nodes);
    const uint64_t* node = X.nodes + (uint64_t)fr.root * 256;
    for (int d = 0; d < 8; ++d) {
        const uint64_t e = __ldg(node + (key >> 56));
        ++*gathers;
        key <<= 8;
        if ((e & 3ull) != 0ull || e == 0ull) return e;
        if ((e >> 11) >= X.n_nodes) { atomicOr((unsigned long long*)err, kErrTrieBounds); return 0; }
        node = reinterpret_cast<const uint64_t*>(base + e);
    }
    atomicOr((unsigned long long*)err, kErrTrieBounds);
    return 0;
}

// The polygon id a join reports for a piece reference.
__device__ __forceinline__ uint32_t out_poly(const DevIndex& X, uint32_t piece) {
    return X.piece_poly ? __ldg(X.piece_poly + piece) : piece;
}

// Number of references (true + candidate) an entry holds.
__device__ __forceinline__ void entry_counts(const DevIndex& X, uint64_t e, uint32_t* n_true, uint32_t* n_cand) {
    const uint32_t tag = (uint32_t)(e & 3ull);
    *n_true = 0;
    *n_cand = 0;
    if (tag == 1) {
        const uint32_t p = (uint32_t)(e >> 2) & 0x7FFFFFFFu;
        if (p == kInvalidPayloadDev) return;
        if (p & 1u) *n_true = 1; else *n_cand = 1;
    } else if (tag == 2) {
        const uint32_t p1 = (uint32_t)(e >> 2) & 0x7FFFFFFFu, p2 = (uint32_t)(e >> 33) & 0x7FFFFFFFu;
        *n_true = (p1 & 1u) + (p2 & 1u);
        *n_cand = 2 - *n_true;
    } else if (tag == 3) {
        const uint32_t off = (uint32_t)(e >> 2) & 0x7FFFFFFFu;
        const uint32_t nt = __ldg(X.lut + off);
        *n_true = nt;
        *n_cand = __ldg(X.lut + off + 1 + nt);
    }
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace agj
