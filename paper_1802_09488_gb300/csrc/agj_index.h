// agj_index.h — host-side index representation shared by the builder (C++)
// and the CUDA front end.  No CUDA types here so that the builder compiles
// with a plain C++ compiler.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/agj.h"
#include "agj_geom.cuh"

namespace agj {

// Tagged 8-byte trie entry (§III-C "Adaptive Cell Trie"):
//   low 2 bits = tag
//   tag 0: child pointer, stored as node_index << 11 (the byte offset of the
//          child's 256 x 8-byte node); the value 0 is the sentinel (false hit)
//   tag 1: one inline payload in bits 2..32
//   tag 2: two inline payloads in bits 2..32 and 33..63
//   tag 3: word offset into the lookup table in bits 2..32
// A payload is polygon_id << 1 | interior (31 bits); 0x7FFFFFFF is the
// invalid payload (false hit).
constexpr uint64_t kTagMask = 3;
constexpr uint64_t kTagPtr = 0, kTagOne = 1, kTagTwo = 2, kTagLut = 3;
constexpr uint32_t kPayloadMask = 0x7FFFFFFFu;
constexpr uint32_t kInvalidPayload = 0x7FFFFFFFu;
constexpr uint32_t kNodeEntries = 256;
constexpr int kNodeShift = 11;               // log2(256 * 8)
constexpr uint32_t kNoRoot = 0xFFFFFFFFu;
constexpr uint32_t kMaxPolys = (1u << 30) - 1;

// Face table entry (§IV-B stage 1: roots, common prefixes, prefix lengths).
// prefix_bits counts key bits after the 3 face bits (a multiple of 8); the
// prefix is right-aligned.
struct FaceRoot {
    uint32_t root;
    uint32_t prefix_bits;
    uint64_t prefix;
};

// The edges of polygon k of X: the first vertex (relative to poly_off[k])
// of every edge; the edge's second vertex is the next one, modulo the
// vertex count for a one-ring polygon.
struct Index;
void poly_edges(const Index& X, uint32_t k, std::vector<uint32_t>* out);

struct Index {
    agj_mode mode = AGJ_APPROX;
    // The index's polygons are pieces: one per cube face an input polygon
    // reaches (most polygons are one piece).  References, geometry and the
    // refine run on pieces; joins and counts report input polygon ids
    // (piece_poly maps them; empty when every polygon is one piece, piece k
    // = polygon k).
    uint32_t n_polys = 0;             // pieces
    uint32_t n_input_polys = 0;       // polygons given to agj_build
    std::vector<uint32_t> piece_poly; // input polygon of each piece (ascending), or empty
    bool contains = false;      // exact join by ST_Contains (boundary points excluded) instead of ST_Covers
    double precision_m = 0;
    // logical index (super covering)
    std::vector<uint64_t> cells;
    std::vector<uint64_t> ref_off;
    std::vector<uint32_t> refs;
    // physical index
    std::vector<uint64_t> nodes;
    std::vector<uint32_t> lut;
    FaceRoot faces[6];
    // polygons in face (u,v)
    std::vector<double> poly_uv;      // 2 per vertex
    std::vector<uint32_t> poly_off;   // n_polys + 1
    // Polygons with holes store every ring explicitly closed (its first
    // vertex repeated at its end), so each of their edges is (t, t + 1);
    // ring_end[ring_off[k] .. ring_off[k+1]) are the ends of polygon k's rings
    // relative to poly_off[k] (none for a one-ring polygon, whose ring is
    // implicitly closed: edge t is (t, t + 1 mod V)).
    std::vector<uint32_t> ring_off;   // n_polys + 1
    std::vector<uint32_t> ring_end;
    std::vector<double> poly_bbox;    // 4 per polygon: umin umax vmin vmax
    std::vector<int8_t> poly_face;
    FastModel model{};                // certified fast cell ids (disabled: all zero)
    std::vector<PolyLocal> poly_local;   // per polygon: reference point, rounding bound, bbox
    std::vector<F2> poly_luv;            // per vertex: FP32 local coordinates
    std::vector<uint16_t> poly_band;     // per polygon: band tables of the certified test
    agj_stats stats{};
    // device copies (owned)
    void* d_blob = nullptr;
    uint64_t blob_bytes = 0;
    uint64_t off_nodes = 0, off_lut = 0, off_uv = 0, off_vkey = 0, off_ukey = 0, off_poff = 0, off_bbox = 0,
             off_face = 0, off_plocal = 0, off_pluv = 0, off_pband = 0, off_roff = 0, off_rend = 0, off_ppoly = 0;
    int device = 0;
};

struct BuildParams {
    agj_mode mode;
    double precision_m;
    uint32_t max_cover_cells, max_cover_level, max_interior_cells, max_interior_level;
    uint64_t budget;
    const double* train;
    uint64_t n_train;
    uint32_t max_train_level;
    uint32_t threads;
    bool fast_ids;
    bool pip_bands;
};

// Host build of the logical and physical index (no CUDA calls).  Returns an
// AGJ_* status; on failure *err_msg says why.
int build_host(const agj_polygon* polys, uint32_t n_polys, const BuildParams& bp, Index* out,
               std::string* err_msg);

// Training (§III-D) of an exact index from the leaf cell ids of training
// points: splits its expensive cells within `budget` node bytes (0: 4x the
// current trie) down to max_level (0: 24), then re-flattens the trie and
// re-fits the fast cell-id model.  Host only; the device copy is not touched.
int retrain(Index* X, const uint64_t* ids, uint64_t n_ids, uint64_t budget, uint32_t max_level, unsigned threads,
            std::string* err);

// Fits idx->model (the certified fast cell-id model) for the index's cells;
// leaves it disabled when the cells span faces or too wide a window.
void fit_fast_model(Index* idx, unsigned threads);

// Local FP32 coordinates of every polygon for the certified refine step.
void prepare_poly_local(Index* idx, bool bands);
// band tables of the certified refine test: at least kBandMinVerts vertices,
// at most kBandMax bands and kBandMaxWords uint16 words per polygon
constexpr uint32_t kBandMinVerts = 24;
constexpr uint32_t kBandMax = 64;
constexpr uint32_t kBandMaxWords = 4096;

// The super-covering merge on given (cell, reference) pairs, in order.
void supercover(const uint64_t* cells, const uint32_t* refs, uint64_t n, std::vector<uint64_t>* out_cells,
                std::vector<uint64_t>* out_off, std::vector<uint32_t>* out_refs);

// Lookup-table encoding of reference lists (deduplicated).
void lut_encode(const uint32_t* refs, const uint64_t* ref_off, uint64_t n_lists, std::vector<uint32_t>* words,
                std::vector<uint64_t>* offsets);

}  // namespace agj
