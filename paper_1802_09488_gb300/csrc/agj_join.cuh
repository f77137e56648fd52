// agj_join.cuh — host side of one join launch sequence over a job source
// (one job for the plain join, many for the batched form): the work-space
// layout and the kernels enqueued on a stream.  Nothing here allocates or
// synchronises, so the sequence can be captured into a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "agj_index.h"
#include "agj_probe.cuh"

namespace agj {

// defined in agj_kernels.cu
int sm_count();
DevIndex make_dev_index(const Index& X);
// A job descriptor of (X, d_points, n, out) with its diagnostics in counters;
// tile0 and poly0 are zero (the plain join's single job).
JobDesc make_job(const Index& X, const double* d_points, uint64_t n, agj_pairs* out, uint64_t* counters);

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Work space of one join launch sequence, as byte offsets into one buffer:
//   [header 256 B: u32 tile-scan chunk counter, u32 unused,
//    u32 refine chunks, u32 polygon-scan chunk counter,
//    u64 FP64 cell-id fallbacks, u64 FP64 refine fallbacks, u64 scan errors]
//   [tile-scan chunk states] [exact: polygon-scan chunk states,
//    per-polygon candidate counts]
//   -- the part zeroed before every launch sequence --
//   [entries u64 per point] [tile counts u32] [tile prefixes u32]
//   then, with exact jobs, the per-tile candidate counts, the candidate
//   queue (a region of tile_slots per tile), its pass bytes, its polygon
//   order, the per-polygon cursors and the refine chunk descriptors
struct JoinLayout {
    uint64_t chunks = 0, pchunks = 0, pcount = 0, stripes = 0, zero_end = 0;
    uint64_t entries = 0, tcount = 0, tprefix = 0;
    uint64_t tcand = 0, queue = 0, pass = 0, sorted = 0, cursor = 0, cpoly = 0, total = 0;
    uint64_t n_points = 0, n_tiles = 0, n_chunks = 0, n_pchunks = 0, queue_cap = 0, n_polys = 0;
    uint32_t tile_slots = 0;
    bool exact = false;
};

constexpr uint64_t kHdrIdFallbacks = 2;    // u64 word of the header
constexpr uint64_t kHdrRefineFallbacks = 3;
constexpr uint64_t kHdrScanErr = 4;
constexpr uint64_t kPolyScanPerCta = 256 * 4;

// n_points / n_tiles: sizes of the (tile-padded) global point space and of
// the tile space; exact: some job refines; tile_slots: queue slots per tile;
// n_polys: polygons of the exact jobs.  count: the aggregation mode's work
// space, which holds no per-point entries, tile counts, prefixes or pass
// bytes (those offsets stay 0 and are not used), and with n_hist_polys
// (polygons counted in shared memory) the zeroed striped histograms.
constexpr uint32_t kAggStripes = 64;
inline JoinLayout join_layout(uint64_t n_points, uint64_t n_tiles, bool exact, uint32_t tile_slots, uint64_t n_polys,
                              bool count = false, uint64_t n_hist_polys = 0) {
    JoinLayout L;
    L.n_points = n_points;
    L.n_tiles = n_tiles;
    L.exact = exact;
    L.n_chunks = (n_tiles + 256 * kScanItems - 1) / (256 * kScanItems);
    uint64_t o = 256;
    L.chunks = o;
    o += align256((L.n_chunks + 1) * 8);        // + 1: the batched form scans its two modes' tiles apart
    if (exact) {
        L.n_polys = n_polys;
        L.tile_slots = tile_slots;
        L.queue_cap = n_tiles * tile_slots;
        L.n_pchunks = (n_polys + kPolyScanPerCta - 1) / kPolyScanPerCta;
        L.pchunks = o;
        o += align256(std::max<uint64_t>(L.n_pchunks, 1) * 8);
        L.pcount = o;
        o += align256(n_polys * 4 + 4);
    }
    if (count && n_hist_polys) {
        // aggregation mode: kAggStripes striped u32 copies of the histogram
        L.stripes = o;
        o += align256((uint64_t)kAggStripes * n_hist_polys * 4);
    }
    L.zero_end = o;
    if (!count) {
        L.entries = o; o += align256(n_points * 8 + 8);
        L.tcount = o; o += align256(n_tiles * 4 + 4);
        L.tprefix = o; o += align256(n_tiles * 4 + 4);
    }
    if (exact) {
        L.tcand = o; o += align256(n_tiles * 4 + 4);
        L.queue = o; o += align256(L.queue_cap * 8 + 8);
        if (!count) { L.pass = o; o += align256(L.queue_cap + 32); }
        L.sorted = o; o += align256(L.queue_cap * 8 + 8);
        L.cursor = o; o += align256((n_polys + 1) * 4);
        // refine chunk descriptors: one per kPipBlock candidates of a polygon, plus one partial per polygon
        L.cpoly = o; o += align256((L.queue_cap / kPipBlock + n_polys + 1) * 16);
    }
    L.total = o;
    return L;
}

inline JoinScratch join_scratch(const JoinLayout& L, char* sc) {
    JoinScratch S;
    S.entries = reinterpret_cast<uint64_t*>(sc + L.entries);
    S.tile_count = reinterpret_cast<uint32_t*>(sc + L.tcount);
    S.tile_prefix = reinterpret_cast<uint32_t*>(sc + L.tprefix);
    S.queue = L.exact ? reinterpret_cast<uint2*>(sc + L.queue) : nullptr;
    S.pass = L.exact ? reinterpret_cast<uint8_t*>(sc + L.pass) : nullptr;
    S.tile_cand = L.exact ? reinterpret_cast<uint32_t*>(sc + L.tcand) : nullptr;
    S.poly_count = L.exact ? reinterpret_cast<uint32_t*>(sc + L.pcount) : nullptr;
    S.tile_slots = L.tile_slots;
    S.scan_err = reinterpret_cast<const uint64_t*>(sc) + kHdrScanErr;
    return S;
}

struct JoinLaunch {
    int probe_grid = 0;       // CTAs of the probe kernel (split form: of the exact tiles' probe)
    int emit_grid = 0;        // CTAs of the emit kernel (split form: of the exact tiles' emit)
    int probe_grid_a = 0;     // split form: CTAs of the approximate tiles' probe
    int emit_grid_a = 0;      // split form: CTAs of the approximate tiles' emit
    int sms = 1;              // for the grid-stride kernels
    bool persistent = false;  // batched form: probe grids smaller than the tile space stride over it
    int pip_grid = 0;
    const uint16_t* tile_job = nullptr;   // batched form: job of each tile
    uint32_t* job_base = nullptr;         // batched form: tile prefix at each job's first tile
};

// Enqueues zeroing, probe, refine (exact jobs), scan and emit.  extra_zero /
// n_extra: further words zeroed by the first kernel (the plain join's status).
// events: null or 4 events recorded before the probe, after the probe, after
// the refine (exact) or the scan (approximate), and at the end.
template <int PPT, class Src, int MODE>
cudaError_t enqueue_join(const Src& src, const JoinLayout& L, char* sc, const JoinLaunch& G, uint64_t* extra_zero,
                         uint64_t n_extra, cudaStream_t s, cudaEvent_t const* events) {
    auto mark = [&](int k) {
        if (events) cudaEventRecord(events[k], s);
    };
    const JoinScratch S = join_scratch(L, sc);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sc);
    {
        const uint64_t zero_words = L.zero_end / 8;
        const int grid = (int)std::min<uint64_t>((zero_words + n_extra + 255) / 256 + 1, (uint64_t)G.sms * 4);
        k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), zero_words, extra_zero, n_extra);
    }
    mark(0);
    if (L.n_tiles) {
        if constexpr (!Src::kSingle) {
            if (G.persistent) {
                k_probe<PPT, Src, MODE, true><<<G.probe_grid, kJoinBlock, 0, s>>>(src, L.n_tiles, S);
            } else {
                k_probe<PPT, Src, MODE><<<G.probe_grid, kJoinBlock, 0, s>>>(src, L.n_tiles, S);
            }
        } else {
            k_probe<PPT, Src, MODE><<<G.probe_grid, kJoinBlock, 0, s>>>(src, L.n_tiles, S);
        }
    }
    mark(1);
    const bool refine = MODE != kModeApprox && L.exact && L.n_polys;
    if (refine && L.n_tiles) {
        const uint32_t ct = refine_chunk_tiles(L.n_tiles, G.sms, L.n_polys);
        k_count<<<refine_sort_grid(L.n_tiles, ct, G.sms, AGJ_COUNT_CTAS_PER_SM), 256, 0, s>>>(
            S.queue, S.tile_cand, L.n_tiles, L.tile_slots, ct, S.poly_count, (uint32_t)L.n_polys);
        k_poly_scan<<<(unsigned)L.n_pchunks, 256, 0, s>>>(
            S.poly_count, (uint32_t)L.n_polys, reinterpret_cast<uint32_t*>(sc + L.cursor), hdr + 2,
            reinterpret_cast<uint4*>(sc + L.cpoly), reinterpret_cast<uint64_t*>(sc + L.pchunks), hdr + 3,
            reinterpret_cast<uint64_t*>(sc) + kHdrScanErr);
        k_scatter<<<refine_sort_grid(L.n_tiles, ct, G.sms, AGJ_SCATTER_CTAS_PER_SM), 256, 0, s>>>(
            S.queue, S.tile_cand, L.n_tiles, L.tile_slots, ct, reinterpret_cast<uint32_t*>(sc + L.cursor),
            reinterpret_cast<uint2*>(sc + L.sorted), (uint32_t)L.n_polys);
        k_pip<Src><<<G.pip_grid, kPipBlock, 0, s>>>(src, 32 * PPT, reinterpret_cast<const uint2*>(sc + L.sorted),
                                                    reinterpret_cast<const uint4*>(sc + L.cpoly), hdr + 2, S.pass,
                                                    S.tile_count);
    }
    if (MODE == kModeApprox) {
        if (L.n_tiles)
            k_scan_counts<<<(unsigned)L.n_chunks, 256, 0, s>>>(S.tile_count, L.n_tiles, S.tile_prefix,
                                                               reinterpret_cast<uint64_t*>(sc + L.chunks), hdr,
                                                               reinterpret_cast<uint64_t*>(sc) + kHdrScanErr,
                                                               G.tile_job, G.job_base);
        mark(2);
    } else {
        mark(2);
        if (L.n_tiles)
            k_scan_counts<<<(unsigned)L.n_chunks, 256, 0, s>>>(S.tile_count, L.n_tiles, S.tile_prefix,
                                                               reinterpret_cast<uint64_t*>(sc + L.chunks), hdr,
                                                               reinterpret_cast<uint64_t*>(sc) + kHdrScanErr,
                                                               G.tile_job, G.job_base);
    }
    if (L.n_tiles) k_emit<PPT, Src, MODE><<<G.emit_grid, kJoinBlock, 0, s>>>(src, L.n_tiles, S);
    mark(3);
    return cudaGetLastError();
}

// The batched form with both modes over many tiles: the approximate tiles
// (0 .. src.ta - 1) and the exact ones (src.ta .. n_tiles - 1) run as two
// independent chains, each with its own probe, scan and emit compiled for
// its mode, the exact one with the refine over its tiles only.  The chains
// share no work space (disjoint tiles, points, queue regions, scan states and
// tickets), so with an auxiliary stream (s_aux, fork and join events) the
// approximate chain runs beside the exact one, e.g. as a parallel branch of
// a captured graph; without one, both run on s in turn.
template <int PPT>
cudaError_t enqueue_join_split(const ManyJobs& src, const JoinLayout& L, char* sc, const JoinLaunch& G,
                               cudaStream_t s, cudaStream_t s_aux, cudaEvent_t fork, cudaEvent_t join) {
    const JoinScratch S = join_scratch(L, sc);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(sc);
    uint64_t* err = reinterpret_cast<uint64_t*>(sc) + kHdrScanErr;
    uint64_t* chunks = reinterpret_cast<uint64_t*>(sc + L.chunks);
    const uint64_t ta = src.ta, T = L.n_tiles;
    {
        const uint64_t zero_words = L.zero_end / 8;
        const int grid = (int)std::min<uint64_t>((zero_words + 255) / 256 + 1, (uint64_t)G.sms * 4);
        k_zero<<<grid, 256, 0, s>>>(reinterpret_cast<uint64_t*>(sc), zero_words, nullptr, 0);
    }
    cudaStream_t sa = s;
    if (s_aux) {
        if (cudaEventRecord(fork, s) != cudaSuccess || cudaStreamWaitEvent(s_aux, fork, 0) != cudaSuccess)
            return cudaGetLastError();
        sa = s_aux;
    }
    const uint64_t per_chunk = 256 * kScanItems;
    const uint64_t na = (ta + per_chunk - 1) / per_chunk, ne = (T - ta + per_chunk - 1) / per_chunk;
    // approximate chain: tiles 0 .. ta - 1, scan ticket hdr[0], chunk states 0 .. na - 1
    {
        ManyJobs a = src;
        a.t0 = 0;
        if (G.persistent) k_probe<PPT, ManyJobs, kModeApprox, true><<<G.probe_grid_a, kJoinBlock, 0, sa>>>(a, ta, S);
        else k_probe<PPT, ManyJobs, kModeApprox><<<G.probe_grid_a, kJoinBlock, 0, sa>>>(a, ta, S);
        k_scan_counts<<<(unsigned)na, 256, 0, sa>>>(S.tile_count, ta, S.tile_prefix, chunks, hdr, err, G.tile_job,
                                                    G.job_base);
        k_emit<PPT, ManyJobs, kModeApprox><<<G.emit_grid_a, kJoinBlock, 0, sa>>>(a, ta, S);
    }
    // exact chain: tiles ta .. T - 1, scan ticket hdr[1], chunk states na .. na + ne - 1
    {
        ManyJobs x = src;
        x.t0 = ta;
        if (G.persistent) k_probe<PPT, ManyJobs, kModeExact, true><<<G.probe_grid, kJoinBlock, 0, s>>>(x, T, S);
        else k_probe<PPT, ManyJobs, kModeExact><<<G.probe_grid, kJoinBlock, 0, s>>>(x, T, S);
        if (L.n_polys) {
            // the refine over the exact tiles' queue regions (slots relative to tile ta)
            const uint64_t q0 = ta * L.tile_slots;
            const uint32_t ct = refine_chunk_tiles(T - ta, G.sms, L.n_polys);
            k_count<<<refine_sort_grid(T - ta, ct, G.sms, AGJ_COUNT_CTAS_PER_SM), 256, 0, s>>>(
                S.queue + q0, S.tile_cand + ta, T - ta, L.tile_slots, ct, S.poly_count, (uint32_t)L.n_polys);
            k_poly_scan<<<(unsigned)L.n_pchunks, 256, 0, s>>>(
                S.poly_count, (uint32_t)L.n_polys, reinterpret_cast<uint32_t*>(sc + L.cursor), hdr + 2,
                reinterpret_cast<uint4*>(sc + L.cpoly), reinterpret_cast<uint64_t*>(sc + L.pchunks), hdr + 3, err);
            k_scatter<<<refine_sort_grid(T - ta, ct, G.sms, AGJ_SCATTER_CTAS_PER_SM), 256, 0, s>>>(
                S.queue + q0, S.tile_cand + ta, T - ta, L.tile_slots, ct, reinterpret_cast<uint32_t*>(sc + L.cursor),
                reinterpret_cast<uint2*>(sc + L.sorted), (uint32_t)L.n_polys);
            k_pip<ManyJobs><<<G.pip_grid, kPipBlock, 0, s>>>(src, 32 * PPT, reinterpret_cast<const uint2*>(sc + L.sorted),
                                                            reinterpret_cast<const uint4*>(sc + L.cpoly), hdr + 2,
                                                            S.pass + q0, S.tile_count);
        }
        k_scan_counts<<<(unsigned)ne, 256, 0, s>>>(S.tile_count + ta, T - ta, S.tile_prefix + ta, chunks + na, hdr + 1,
                                                   err, G.tile_job + ta, G.job_base);
        k_emit<PPT, ManyJobs, kModeExact><<<G.emit_grid, kJoinBlock, 0, s>>>(x, T, S);
    }
    if (s_aux) {
        if (cudaEventRecord(join, s_aux) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess)
            return cudaGetLastError();
    }
    return cudaGetLastError();
}

}  // namespace agj
