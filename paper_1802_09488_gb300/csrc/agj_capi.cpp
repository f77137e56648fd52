// agj_capi.cpp — the extern "C" boundary declared in include/agj.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/agj.h"
#include "agj_geom.cuh"
#include "agj_handle.h"
#include "agj_index.h"
#include "agj_launch.h"

struct agj_batch {
    agj::Batch* B;
};

namespace {

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// The address kernels on the current device read host buffer p through, or
// null: pinned (registered) memory through its device mapping, pageable
// memory where the device reads the host's page tables; 16-byte aligned
// buffers only (the probe loads 16-byte points).
const void* device_view(const void* p) {
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u) != 0) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    int dev = 0, pageable = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return pageable == 1 ? p : nullptr;
}

thread_local std::string g_last_error;

}  // namespace

extern "C" {

const char* agj_strerror(int status) {
    switch (status) {
        case AGJ_OK: return "ok";
        case AGJ_EINVAL: return "invalid argument";
        case AGJ_EUNSUPPORTED: return "unsupported input";
        case AGJ_EBUDGET: return "memory budget exceeded";
        case AGJ_ENOMEM: return "out of memory";
        case AGJ_ECUDA: return "CUDA error";
        case AGJ_ETIMEOUT: return "device wait timed out";
        case AGJ_EBUSY: return "busy";
        case AGJ_ECAPACITY: return "buffer too small";
        case AGJ_EDEVICE: return "device-side check failed";
        default: return "unknown status";
    }
}

// Last build error message of the calling thread (diagnostics only).
const char* agj_last_error(void) { return g_last_error.c_str(); }

int agj_build(const agj_polygon* polys, uint32_t n_polys, double precision_m, agj_mode mode,
              const agj_build_opts* opts, void* stream, agj_index** out) {
    if (!out) return AGJ_EINVAL;
    *out = nullptr;
    if (mode != AGJ_APPROX && mode != AGJ_EXACT && mode != AGJ_AUTO) return AGJ_EINVAL;
    agj_build_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (o.predicate > AGJ_CONTAINS) return AGJ_EINVAL;
    if (mode == AGJ_AUTO) {
        // §III-A: the approximate index first; if it exceeds the memory
        // budget, the exact index, trained until the budget is spent
        if (!o.memory_budget_bytes) return AGJ_EINVAL;
        const int rc = agj_build(polys, n_polys, precision_m, AGJ_APPROX, &o, stream, out);
        if (rc != AGJ_EBUDGET) return rc;
        return agj_build(polys, n_polys, precision_m, AGJ_EXACT, &o, stream, out);
    }
    agj::BuildParams bp;
    bp.mode = mode;
    bp.precision_m = precision_m;
    bp.max_cover_cells = o.max_cover_cells ? o.max_cover_cells : 128;
    bp.max_cover_level = o.max_cover_level ? std::min<uint32_t>(o.max_cover_level, 30) : 30;
    bp.max_interior_cells = o.max_interior_cells ? o.max_interior_cells : 256;
    bp.max_interior_level = o.max_interior_level ? std::min<uint32_t>(o.max_interior_level, 30) : 20;
    bp.budget = o.memory_budget_bytes;
    bp.train = o.train_latlng;
    bp.n_train = o.train_latlng ? o.n_train : 0;
    bp.max_train_level = o.max_train_level ? std::min<uint32_t>(o.max_train_level, 30) : 24;
    bp.threads = o.n_threads;
    bp.fast_ids = !o.no_fast_ids;
    bp.pip_bands = !o.no_pip_bands;
    agj_index* h = new (std::nothrow) agj_index();
    if (!h) return AGJ_ENOMEM;
    int rc;
    try {
        rc = agj::build_host(polys, n_polys, bp, &h->X, &g_last_error);
    } catch (const std::bad_alloc&) {
        rc = AGJ_ENOMEM;
    }
    if (rc == AGJ_OK) {
        h->X.stats.predicate = o.predicate;
        h->X.contains = o.predicate == AGJ_CONTAINS;
    }
    if (rc == AGJ_OK && !o.host_only) rc = agj::upload_index(&h->X, as_stream(stream));
    if (rc != AGJ_OK) {
        agj_free(h);
        return rc;
    }
    *out = h;
    return AGJ_OK;
}

void agj_free(agj_index* index) {
    if (!index) return;
    if (index->X.d_blob) {
        cudaDeviceSynchronize();
        cudaFree(index->X.d_blob);
    }
    delete index;
}

int agj_index_stats(const agj_index* index, agj_stats* out) {
    if (!index || !out) return AGJ_EINVAL;
    *out = index->X.stats;
    return AGJ_OK;
}

int agj_index_logical(const agj_index* index, uint64_t* cells, uint64_t* ref_off, uint32_t* refs, uint64_t* n_cells,
                      uint64_t* n_refs) {
    if (!index) return AGJ_EINVAL;
    const agj::Index& X = index->X;
    if (n_cells) *n_cells = X.cells.size();
    if (n_refs) *n_refs = X.refs.size();
    if (cells) std::copy(X.cells.begin(), X.cells.end(), cells);
    if (ref_off) std::copy(X.ref_off.begin(), X.ref_off.end(), ref_off);
    if (refs) {
        // references name input polygons (the index refers to pieces; a cell
        // lies on one face, so it holds at most one piece of a polygon)
        if (X.piece_poly.empty()) {
            std::copy(X.refs.begin(), X.refs.end(), refs);
        } else {
            for (size_t t = 0; t < X.refs.size(); ++t)
                refs[t] = X.piece_poly[X.refs[t] >> 1] << 1 | (X.refs[t] & 1u);
        }
    }
    return AGJ_OK;
}

int agj_supercover(const uint64_t* cells, const uint32_t* refs, uint64_t n, uint64_t* out_cells, uint64_t* out_off,
                   uint32_t* out_refs, uint64_t* n_out_cells, uint64_t* n_out_refs) {
    if (n && (!cells || !refs)) return AGJ_EINVAL;
    for (uint64_t k = 0; k < n; ++k) {
        // a cell id: face <= 5 and its lowest set (marker) bit at an even position
        if (cells[k] == 0 || (cells[k] >> 61) > 5 || (__builtin_ctzll(cells[k]) & 1)) return AGJ_EINVAL;
    }
    std::vector<uint64_t> oc, oo;
    std::vector<uint32_t> orf;
    agj::supercover(cells, refs, n, &oc, &oo, &orf);
    if (n_out_cells) *n_out_cells = oc.size();
    if (n_out_refs) *n_out_refs = orf.size();
    if (out_cells) std::copy(oc.begin(), oc.end(), out_cells);
    if (out_off) std::copy(oo.begin(), oo.end(), out_off);
    if (out_refs) std::copy(orf.begin(), orf.end(), out_refs);
    return AGJ_OK;
}

int agj_lut_encode(const uint32_t* refs, const uint64_t* ref_off, uint64_t n_lists, uint32_t* words,
                   uint64_t* offsets, uint64_t* n_words) {
    if (n_lists && (!refs || !ref_off)) return AGJ_EINVAL;
    std::vector<uint32_t> w;
    std::vector<uint64_t> o;
    agj::lut_encode(refs, ref_off, n_lists, &w, &o);
    if (n_words) *n_words = w.size();
    if (words) std::copy(w.begin(), w.end(), words);
    if (offsets) std::copy(o.begin(), o.end(), offsets);
    return AGJ_OK;
}

int agj_index_trie(const agj_index* index, uint64_t* nodes, uint32_t* lut, uint64_t face_table[18]) {
    if (!index) return AGJ_EINVAL;
    const agj::Index& X = index->X;
    if (nodes) std::copy(X.nodes.begin(), X.nodes.end(), nodes);
    if (lut) std::copy(X.lut.begin(), X.lut.end(), lut);
    if (face_table)
        for (int f = 0; f < 6; ++f) {
            face_table[3 * f] = X.faces[f].root;
            face_table[3 * f + 1] = X.faces[f].prefix_bits;
            face_table[3 * f + 2] = X.faces[f].prefix;
        }
    return AGJ_OK;
}

int agj_join_requirements(const agj_index* index, uint64_t n, agj_requirements* out) {
    if (!index || !out) return AGJ_EINVAL;
    return agj::join_requirements(index->X, n, out);
}

int agj_pairs_alloc(const agj_index* index, uint64_t n, void* stream, agj_pairs* out) {
    if (!index || !out) return AGJ_EINVAL;
    agj_requirements r;
    agj::join_requirements(index->X, n, &r);
    memset(out, 0, sizeof *out);
    cudaStream_t s = as_stream(stream);
    void *off = nullptr, *ids = nullptr, *scr = nullptr, *st = nullptr;
    if (cudaMallocAsync(&off, (n + 1) * 4, s) != cudaSuccess ||
        cudaMallocAsync(&ids, std::max<uint64_t>(r.ids_capacity, 1) * 4, s) != cudaSuccess ||
        cudaMallocAsync(&scr, r.scratch_bytes, s) != cudaSuccess || cudaMallocAsync(&st, 64, s) != cudaSuccess) {
        cudaGetLastError();
        if (off) cudaFreeAsync(off, s);
        if (ids) cudaFreeAsync(ids, s);
        if (scr) cudaFreeAsync(scr, s);
        if (st) cudaFreeAsync(st, s);
        return AGJ_ENOMEM;
    }
    out->offsets = static_cast<uint32_t*>(off);
    out->ids = static_cast<uint32_t*>(ids);
    out->ids_capacity = r.ids_capacity;
    out->scratch = scr;
    out->scratch_bytes = r.scratch_bytes;
    out->status = static_cast<uint64_t*>(st);
    return AGJ_OK;
}

int agj_pairs_free(agj_pairs* pairs, void* stream) {
    if (!pairs) return AGJ_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (pairs->offsets) cudaFreeAsync(pairs->offsets, s);
    if (pairs->ids) cudaFreeAsync(pairs->ids, s);
    if (pairs->scratch) cudaFreeAsync(pairs->scratch, s);
    if (pairs->status) cudaFreeAsync(pairs->status, s);
    memset(pairs, 0, sizeof *pairs);
    return cudaGetLastError() == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

int agj_join(const agj_index* index, const double* d_points, uint64_t n, void* stream, agj_pairs* out) {
    if (!index || !index->X.d_blob) return AGJ_EINVAL;
    return agj::launch_join(index->X, d_points, n, as_stream(stream), out);
}

int agj_join_timed(const agj_index* index, const double* d_points, uint64_t n, void* stream, agj_pairs* out,
                   void* const events[4]) {
    if (!index || !index->X.d_blob || !events) return AGJ_EINVAL;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) {
        if (!events[k]) return AGJ_EINVAL;
        ev[k] = static_cast<cudaEvent_t>(events[k]);
    }
    return agj::launch_join(index->X, d_points, n, as_stream(stream), out, ev);
}

int agj_join_approx_noalloc(const agj_index* index, const double* d_points, uint64_t n, uint32_t* d_offsets,
                            uint32_t* d_ids, uint64_t ids_capacity, uint64_t* d_status, void* stream) {
    if (!index) return AGJ_EINVAL;
    return agj::launch_join_approx_noalloc(index->X, d_points, n, d_offsets, d_ids, ids_capacity, d_status,
                                           as_stream(stream));
}

uint64_t agj_count_scratch_bytes(const agj_index* index, uint64_t n) {
    return index ? agj::count_scratch_bytes(index->X, n) : 0;
}

int agj_join_count(const agj_index* index, const double* d_points, uint64_t n, void* stream, uint64_t* d_counts,
                   int accumulate, uint64_t* d_status, void* d_scratch, uint64_t scratch_bytes) {
    if (!index || !index->X.d_blob) return AGJ_EINVAL;
    return agj::launch_join_count(index->X, d_points, n, as_stream(stream), d_counts, d_status, d_scratch,
                                  scratch_bytes, accumulate != 0);
}

int agj_join_count_timed(const agj_index* index, const double* d_points, uint64_t n, void* stream, uint64_t* d_counts,
                         int accumulate, uint64_t* d_status, void* d_scratch, uint64_t scratch_bytes,
                         void* const events[4]) {
    if (!index || !index->X.d_blob || !events) return AGJ_EINVAL;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) {
        if (!events[k]) return AGJ_EINVAL;
        ev[k] = static_cast<cudaEvent_t>(events[k]);
    }
    return agj::launch_join_count(index->X, d_points, n, as_stream(stream), d_counts, d_status, d_scratch,
                                  scratch_bytes, accumulate != 0, ev);
}

int agj_train_online(agj_index* index, const double* d_points, uint64_t n, uint64_t memory_budget_bytes,
                     void* stream) {
    if (!index || !index->X.d_blob || (n && !d_points)) return AGJ_EINVAL;
    agj::Index& X = index->X;
    if (X.mode != AGJ_EXACT || (reinterpret_cast<uintptr_t>(d_points) & 15u) != 0 || n >= 0xFFFFFFFFull)
        return AGJ_EINVAL;
    cudaStream_t s = as_stream(stream);
    std::vector<uint64_t> ids;
    if (n) {
        // device pass: the points that land in expensive cells
        char* d = nullptr;
        const uint64_t bytes = 64 + n * 8;
        if (cudaMallocAsync(reinterpret_cast<void**>(&d), bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return AGJ_ENOMEM;
        }
        uint64_t* d_hdr = reinterpret_cast<uint64_t*>(d);            // [0] count, [1..4] status words
        uint64_t* d_out = reinterpret_cast<uint64_t*>(d + 64);
        int rc = cudaMemsetAsync(d, 0, 64, s) == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
        if (rc == AGJ_OK) rc = agj::launch_collect_expensive(X, d_points, n, d_out, d_hdr, d_hdr + 1, s);
        uint64_t hdr[5] = {0, 0, 0, 0, 0};
        if (rc == AGJ_OK && (cudaMemcpyAsync(hdr, d, 40, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                             cudaStreamSynchronize(s) != cudaSuccess))
            rc = AGJ_ECUDA;
        if (rc == AGJ_OK && (hdr[2] & 4ull)) rc = AGJ_EDEVICE;
        if (rc == AGJ_OK) {
            ids.resize(std::min<uint64_t>(hdr[0], n));
            if (!ids.empty() && (cudaMemcpyAsync(ids.data(), d_out, ids.size() * 8, cudaMemcpyDeviceToHost, s) !=
                                     cudaSuccess ||
                                 cudaStreamSynchronize(s) != cudaSuccess))
                rc = AGJ_ECUDA;
        }
        cudaFreeAsync(d, s);
        if (rc != AGJ_OK) { cudaGetLastError(); return rc; }
    }
    // host: split the expensive cells, re-flatten, re-upload
    int rc;
    try {
        rc = agj::retrain(&X, ids.data(), ids.size(), memory_budget_bytes, 0, 0, &g_last_error);
    } catch (const std::bad_alloc&) {
        rc = AGJ_ENOMEM;
    }
    if (rc != AGJ_OK) return rc;
    cudaStreamSynchronize(s);
    void* old = X.d_blob;
    X.d_blob = nullptr;
    rc = agj::upload_index(&X, s);
    if (rc == AGJ_ENOMEM) {          // room for one copy only: drop the old one first
        cudaDeviceSynchronize();
        cudaFree(old);
        old = nullptr;
        rc = agj::upload_index(&X, s);
    }
    if (old) {
        cudaDeviceSynchronize();
        cudaFree(old);
    }
    return rc;
}

int agj_measure_fp64_rate(void* stream, double* flops_per_s) {
    return agj::measure_fp64_rate(as_stream(stream), flops_per_s);
}

int agj_join_check(const agj_pairs* pairs, void* stream, uint64_t* nnz) {
    if (!pairs || !pairs->status) return AGJ_EINVAL;
    uint64_t st[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(st, pairs->status, sizeof st, cudaMemcpyDeviceToHost, as_stream(stream)) != cudaSuccess)
        return AGJ_ECUDA;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return AGJ_ECUDA;
    if (nnz) *nnz = st[0];
    if (st[1] & 1ull) return AGJ_ECAPACITY;
    if (st[1] & 2ull) return AGJ_ETIMEOUT;
    if (st[1] & 4ull) return AGJ_EDEVICE;
    if (st[1] & 8ull) return AGJ_ECAPACITY;
    return AGJ_OK;
}

int agj_batch_create(const agj_index* const* indexes, const uint64_t* n, uint32_t m, const agj_batch_opts* opts,
                     agj_batch** out) {
    if (!out || (m && (!indexes || !n))) return AGJ_EINVAL;
    *out = nullptr;
    std::vector<const agj::Index*> xs(m);
    for (uint32_t j = 0; j < m; ++j) {
        if (!indexes[j]) return AGJ_EINVAL;
        xs[j] = &indexes[j]->X;
    }
    agj_batch_opts o{};
    if (opts) o = *opts;
    agj_batch* h = new (std::nothrow) agj_batch();
    if (!h) return AGJ_ENOMEM;
    const int rc = agj::batch_create(xs.data(), n, m, (int)o.points_per_lane, (int)o.ctas_per_sm, o.no_graph == 0,
                                     &h->B);
    if (rc != AGJ_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return AGJ_OK;
}

int agj_batch_run(agj_batch* batch, const double* const* d_points, void* stream, agj_pairs* outs) {
    if (!batch) return AGJ_EINVAL;
    return agj::batch_run(batch->B, d_points, as_stream(stream), outs);
}

uint64_t agj_batch_device_bytes(const agj_batch* batch) { return batch ? agj::batch_device_bytes(batch->B) : 0; }

void agj_batch_free(agj_batch* batch) {
    if (!batch) return;
    agj::batch_free(batch->B);
    delete batch;
}

int agj_join_batched(const agj_index* const* indexes, const double* const* d_points, const uint64_t* n,
                     uint32_t m, void* stream, agj_pairs* outs) {
    agj_batch* b = nullptr;
    int rc = agj_batch_create(indexes, n, m, nullptr, &b);
    if (rc != AGJ_OK) return rc;
    rc = agj_batch_run(b, d_points, stream, outs);
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess && rc == AGJ_OK) rc = AGJ_ECUDA;
    agj_batch_free(b);
    return rc;
}

int agj_join_host(const agj_index* index, const double* h_points, uint64_t n, double* d_points_staging,
                  agj_pairs* work, uint32_t* h_offsets, uint32_t* h_ids, uint64_t h_ids_capacity, uint64_t* nnz,
                  void* stream) {
    if (!index || !index->X.d_blob || !work || !h_offsets || (n && !h_points)) return AGJ_EINVAL;
    cudaStream_t s = as_stream(stream);
    // the probe reads the points where they are when the device can
    // (pinned memory, or pageable memory read through the host's page
    // tables); otherwise they are copied to the staging buffer first
    const double* src = n ? static_cast<const double*>(device_view(h_points)) : nullptr;
    if (n && !src) {
        if (!d_points_staging) return AGJ_EINVAL;
        if (cudaMemcpyAsync(d_points_staging, h_points, n * 16, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return AGJ_ECUDA;
        src = d_points_staging;
    }
    int rc = agj::launch_join(index->X, src, n, s, work);
    if (rc != AGJ_OK) return rc;
    if (cudaMemcpyAsync(h_offsets, work->offsets, (n + 1) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AGJ_ECUDA;
    uint64_t total = 0;
    rc = agj_join_check(work, stream, &total);
    if (nnz) *nnz = total;
    if (rc != AGJ_OK) return rc;
    if (total > h_ids_capacity) return AGJ_ECAPACITY;
    if (total && cudaMemcpyAsync(h_ids, work->ids, total * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AGJ_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? AGJ_OK : AGJ_ECUDA;
}

int agj_selftest_scan_timeout(void* stream) { return agj::selftest_scan_timeout(as_stream(stream)); }

int agj_selftest_ready_timeout(void* stream) { return agj::selftest_ready_timeout(as_stream(stream)); }

int agj_cell_ids(const double* d_points, uint64_t n, uint64_t* d_ids, void* stream) {
    if (n && (!d_points || !d_ids)) return AGJ_EINVAL;
    return agj::launch_cell_ids(d_points, n, d_ids, as_stream(stream));
}

int agj_fast_ids_host(const agj_index* index, const double* h_points, uint64_t n, uint64_t* h_ids,
                      uint8_t* h_levels) {
    if (!index || (n && (!h_points || !h_ids || !h_levels))) return AGJ_EINVAL;
    const agj::FastModel& M = index->X.model;
    if (!M.enabled) return AGJ_EUNSUPPORTED;
    uint16_t lut[1024];
    for (uint32_t t = 0; t < 1024; ++t) lut[t] = agj::hilbert_lut_entry(t);
    for (uint64_t k = 0; k < n; ++k) {
        uint32_t i, j;
        int lc;
        if (!agj::model_ij(M, h_points[2 * k], h_points[2 * k + 1], &i, &j, &lc)) {
            h_ids[k] = 0;
            h_levels[k] = 255;
            continue;
        }
        h_ids[k] = agj::cell_id_lut(lut, M.face, i, j);
        h_levels[k] = (uint8_t)lc;
    }
    return AGJ_OK;
}

int agj_covers_certified_host(const agj_index* index, const double* h_points, const uint32_t* h_polys, uint64_t n,
                              int8_t* h_out) {
    if (!index || (n && (!h_points || !h_polys || !h_out))) return AGJ_EINVAL;
    const agj::Index& X = index->X;
    for (uint64_t k = 0; k < n; ++k) {
        if (h_polys[k] >= X.n_input_polys) return AGJ_EINVAL;
        // the polygon's piece on the point's face (one piece: the polygon)
        uint32_t poly = h_polys[k];
        if (!X.piece_poly.empty()) {
            double u, v;
            const int f = agj::point_valid(h_points[2 * k], h_points[2 * k + 1])
                              ? agj::face_uv(h_points[2 * k], h_points[2 * k + 1], &u, &v) : -1;
            poly = 0xFFFFFFFFu;
            for (uint32_t q = 0; q < X.n_polys; ++q)
                if (X.piece_poly[q] == h_polys[k] && X.poly_face[q] == f) poly = q;
            if (poly == 0xFFFFFFFFu) { h_out[k] = 0; continue; }
        }
        const agj::PolyLocal& L = X.poly_local[poly];
        const uint32_t v0 = X.poly_off[poly], V = X.poly_off[poly + 1] - v0;
        float pu, pv, dp;
        int r = -1;
        if (L.ok && agj::model_uv_local(X.model, h_points[2 * k], h_points[2 * k + 1], L, &pu, &pv, &dp))
            r = agj::covers_certified(X.poly_luv.data() + v0, V, L, L.nb ? X.poly_band.data() + L.band : nullptr,
                                      pu, pv, dp);
        h_out[k] = (int8_t)r;
    }
    return AGJ_OK;
}

int agj_cell_ids_host(const double* h_points, uint64_t n, uint64_t* h_ids) {
    if (n && (!h_points || !h_ids)) return AGJ_EINVAL;
    for (uint64_t k = 0; k < n; ++k) h_ids[k] = agj::point_cell_id(h_points[2 * k], h_points[2 * k + 1]);
    return AGJ_OK;
}

}  // extern "C"
