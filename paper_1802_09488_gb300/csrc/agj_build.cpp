// agj_build.cpp — host build of the logical index (super covering) and the
// physical index (Adaptive Cell Trie + lookup table).
//
//   coverings          own quadtree coverer over face (u,v) cell rectangles
//                      (the paper uses S2's RegionCoverer, §II, with the §V
//                      defaults 128 covering cells / level 30, 256 interior
//                      cells / level 20)
//   super covering     Listing "Build super covering" (§III-B): duplicates
//                      merge references, an ancestor/descendant conflict is
//                      replaced by the descendant plus the difference cells,
//                      each carrying the ancestor's references
//   approx refinement  §III-A: candidate cells are replaced by their children
//                      until the largest candidate cell's diagonal is below
//                      the precision
//   training           §III-D: cells hit by training points that carry a
//                      candidate reference are split into their four children,
//                      each classified against the referenced polygons, until
//                      the memory budget is spent
//   flattening         §III-C: 256-ary trie, cells denormalised to levels that
//                      are multiples of 4, face table with common prefixes,
//                      1 or 2 references inlined, otherwise a lookup-table
//                      offset; unique lists stored once
//
// Cell classification against a polygon uses the cell's (u,v) rectangle
// widened by kMargin: a widened rectangle met by no polygon edge is wholly
// inside or wholly outside (decided at its centre), otherwise it is a
// boundary (candidate) cell.  kMargin is far above the rounding error of the
// point -> (u,v) -> (s,t) -> (i,j) map, so every point whose id lies in a
// cell has (u,v) inside the widened rectangle.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "agj_geom.cuh"
#include "agj_index.h"

namespace agj {
namespace {

constexpr double kMargin = 1e-12;
constexpr double kCapCos = 0.96592582628906831;       // cos 15 degrees: a cross-face polygon's extent
constexpr double kCapFaceCos = 0.34611705707749302;   // cos 69.75 degrees: faces such a polygon can reach
constexpr double kEarthR = 6371008.8;
constexpr double kDiagSlack = 2e-5;   // metres: widened-rectangle allowance in the precision test

enum : int { kOutside = 0, kInside = 1, kBoundary = 2 };

struct Poly {
    int face;
    const double* uv;   // 2 per vertex
    uint32_t nv;
    double bb[4];       // umin umax vmin vmax
    // edges of a polygon with holes (first vertices; the second is the next
    // vertex, rings stored explicitly closed); null: one ring, every vertex
    // starts an edge and the last one's edge closes the ring
    const uint32_t* edges = nullptr;
    uint32_t n_edges = 0;
    uint32_t edge_count() const { return edges ? n_edges : nv; }
    uint32_t edge(uint32_t q) const { return edges ? edges[q] : q; }
};

struct Rect {
    double u0, u1, v0, v1;
};

struct CellIJ {
    int face, level;
    uint32_t i, j;
};

CellIJ decode(uint64_t id) {
    CellIJ c;
    c.face = (int)(id >> 61);
    c.level = cell_level(id);
    uint32_t o = (uint32_t)c.face & 1u, i = 0, j = 0;
    for (int l = 1; l <= c.level; ++l) {
        const uint32_t d = (uint32_t)((id >> (61 - 2 * l)) & 3ull);
        uint32_t ib = d >> 1, jb = (d >> 1) ^ (d & 1u);
        if (o & 2u) { ib ^= 1u; jb ^= 1u; }
        if (o & 1u) { const uint32_t t = ib; ib = jb; jb = t; }
        i = (i << 1) | ib;
        j = (j << 1) | jb;
        if (d == 0u) o ^= 1u;
        else if (d == 3u) o ^= 3u;
    }
    c.i = i;
    c.j = j;
    return c;
}

Rect cell_rect(uint64_t id) {
    const CellIJ c = decode(id);
    const double sc = std::ldexp(1.0, -c.level);
    return Rect{st_to_uv(c.i * sc), st_to_uv((c.i + 1) * sc), st_to_uv(c.j * sc), st_to_uv((c.j + 1) * sc)};
}

inline Rect widen(const Rect& r, double m) { return Rect{r.u0 - m, r.u1 + m, r.v0 - m, r.v1 + m}; }

inline uint64_t child_id(uint64_t id, int k) {
    const uint64_t lsb = cell_lsb(id);
    return id - lsb + (lsb >> 2) * (2ull * (uint64_t)k + 1ull);
}

// Separating-axis test of a closed segment against a closed rectangle.
inline bool seg_meets_rect(const double* a, const double* b, const Rect& r) {
    if (std::max(a[0], b[0]) < r.u0 || std::min(a[0], b[0]) > r.u1) return false;
    if (std::max(a[1], b[1]) < r.v0 || std::min(a[1], b[1]) > r.v1) return false;
    const double du = b[0] - a[0], dv = b[1] - a[1];
    const double o1 = du * (r.v0 - a[1]) - dv * (r.u0 - a[0]);
    const double o2 = du * (r.v0 - a[1]) - dv * (r.u1 - a[0]);
    const double o3 = du * (r.v1 - a[1]) - dv * (r.u0 - a[0]);
    const double o4 = du * (r.v1 - a[1]) - dv * (r.u1 - a[0]);
    if (o1 > 0 && o2 > 0 && o3 > 0 && o4 > 0) return false;
    if (o1 < 0 && o2 < 0 && o3 < 0 && o4 < 0) return false;
    return true;
}

// ST_Covers ring rule in (u,v): on-edge -> covered; otherwise odd number of
// half-open crossings of the ray towards +u.
// With holes the rule runs over the edges of every ring: on an edge of any
// ring -> covered; otherwise an odd number of crossings in all -> covered.
bool ring_covers(const Poly& P, double pu, double pv) {
    if (!(pu >= P.bb[0] && pu <= P.bb[1] && pv >= P.bb[2] && pv <= P.bb[3])) return false;
    bool inside = false;
    const uint32_t n = P.nv;
    for (uint32_t q = 0, m = P.edge_count(); q < m; ++q) {
        const uint32_t k = P.edge(q);
        const double* a = P.uv + 2 * k;
        const double* b = P.uv + 2 * (k + 1 == n ? 0 : k + 1);
        const double vlo = std::min(a[1], b[1]), vhi = std::max(a[1], b[1]);
        if (pv < vlo || pv > vhi) continue;
        const double o = (b[0] - a[0]) * (pv - a[1]) - (b[1] - a[1]) * (pu - a[0]);
        if (o == 0.0 && pu >= std::min(a[0], b[0]) && pu <= std::max(a[0], b[0])) return true;
        if ((a[1] <= pv && pv < b[1] && o > 0.0) || (b[1] <= pv && pv < a[1] && o < 0.0)) inside = !inside;
    }
    return inside;
}

// Classifies the widened rectangle of `id` against polygon P, looking only
// at `edges` (all edges when null); out_edges receives the edges that meet
// the widened rectangle.
int classify(const Poly& P, uint64_t id, const std::vector<uint32_t>* edges, std::vector<uint32_t>* out_edges) {
    if ((int)(id >> 61) != P.face) return kOutside;
    const Rect r = cell_rect(id);
    const Rect w = widen(r, kMargin);
    out_edges->clear();
    if (w.u1 < P.bb[0] || w.u0 > P.bb[1] || w.v1 < P.bb[2] || w.v0 > P.bb[3]) return kOutside;
    const uint32_t n = P.nv;
    auto test = [&](uint32_t k) {
        const double* a = P.uv + 2 * k;
        const double* b = P.uv + 2 * (k + 1 == n ? 0 : k + 1);
        if (seg_meets_rect(a, b, w)) out_edges->push_back(k);
    };
    if (edges) {
        for (uint32_t k : *edges) test(k);
    } else {
        for (uint32_t q = 0, m = P.edge_count(); q < m; ++q) test(P.edge(q));
    }
    if (!out_edges->empty()) return kBoundary;
    return ring_covers(P, 0.5 * (r.u0 + r.u1), 0.5 * (r.v0 + r.v1)) ? kInside : kOutside;
}

void unit_xyz(int face, double u, double v, double p[3]) {
    face_uv_to_xyz(face, u, v, p);
    const double n = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    p[0] /= n; p[1] /= n; p[2] /= n;
}

double arc_m(const double a[3], const double b[3]) {
    const double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    return kEarthR * std::atan2(std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]),
                                a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
}

double cell_diag_m(uint64_t id) {
    const Rect r = cell_rect(id);
    const int f = (int)(id >> 61);
    double p00[3], p11[3], p01[3], p10[3];
    unit_xyz(f, r.u0, r.v0, p00);
    unit_xyz(f, r.u1, r.v1, p11);
    unit_xyz(f, r.u0, r.v1, p01);
    unit_xyz(f, r.u1, r.v0, p10);
    return std::max(arc_m(p00, p11), arc_m(p01, p10));
}

template <class F>
void parallel_for(size_t n, unsigned threads, F&& fn) {
    if (n == 0) return;
    threads = std::max(1u, std::min<unsigned>(threads, (unsigned)std::min<size_t>(n, 1024)));
    if (threads == 1) {
        for (size_t k = 0; k < n; ++k) fn(k, 0u);
        return;
    }
    std::atomic<size_t> next(0);
    const size_t chunk = std::max<size_t>(1, n / (threads * 16));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < threads; ++t) {
        th.emplace_back([&, t] {
            for (;;) {
                const size_t lo = next.fetch_add(chunk);
                if (lo >= n) break;
                const size_t hi = std::min(n, lo + chunk);
                for (size_t k = lo; k < hi; ++k) fn(k, t);
            }
        });
    }
    for (auto& x : th) x.join();
}

// ---------------------------------------------------------------------------
// per-polygon coverings
// ---------------------------------------------------------------------------

struct QItem {
    uint64_t id;
    std::vector<uint32_t> edges;
};

struct QOrder {
    bool operator()(const QItem* a, const QItem* b) const {
        const int la = cell_level(a->id), lb = cell_level(b->id);
        if (la != lb) return la > lb;   // min-heap on level: largest cells first
        return a->id > b->id;
    }
};

// The <= 4 cells of one level covering the polygon's (widened) bbox.
void start_cells(const Poly& P, std::vector<uint64_t>* out) {
    const double m = 1e-9;
    const uint32_t i0 = st_to_ij(uv_to_st(std::max(-1.0, P.bb[0] - m)));
    const uint32_t i1 = st_to_ij(uv_to_st(std::min(1.0, P.bb[1] + m)));
    const uint32_t j0 = st_to_ij(uv_to_st(std::max(-1.0, P.bb[2] - m)));
    const uint32_t j1 = st_to_ij(uv_to_st(std::min(1.0, P.bb[3] + m)));
    int L = kLevels;
    while (L > 0 && (((i1 >> (kLevels - L)) - (i0 >> (kLevels - L))) > 1 ||
                     ((j1 >> (kLevels - L)) - (j0 >> (kLevels - L))) > 1))
        --L;
    out->clear();
    for (uint32_t ii = i0 >> (kLevels - L); ii <= (i1 >> (kLevels - L)); ++ii)
        for (uint32_t jj = j0 >> (kLevels - L); jj <= (j1 >> (kLevels - L)); ++jj)
            out->push_back(cell_id_from_ij(P.face, ii, jj, L));
}

// Covering: cells that together cover the polygon, at most max_cells
// (boundary cells are split largest-first while the count allows).
void covering(const Poly& P, uint32_t max_cells, int max_level, std::vector<uint64_t>* out) {
    std::vector<uint64_t> start;
    start_cells(P, &start);
    std::vector<QItem*> owned;
    std::priority_queue<QItem*, std::vector<QItem*>, QOrder> pq;
    std::vector<uint32_t> tmp;
    out->clear();
    size_t count = 0;
    for (uint64_t c : start) {
        const int cls = classify(P, c, nullptr, &tmp);
        if (cls == kInside) { out->push_back(c); ++count; }
        else if (cls == kBoundary) { owned.push_back(new QItem{c, tmp}); pq.push(owned.back()); ++count; }
    }
    while (!pq.empty()) {
        QItem* q = pq.top();
        pq.pop();
        if (cell_level(q->id) >= max_level) { out->push_back(q->id); continue; }
        QItem* kids[4];
        int cls[4], nk = 0;
        for (int k = 0; k < 4; ++k) {
            const uint64_t c = child_id(q->id, k);
            cls[k] = classify(P, c, &q->edges, &tmp);
            kids[k] = nullptr;
            if (cls[k] != kOutside) { kids[k] = new QItem{c, tmp}; ++nk; }
        }
        if (count - 1 + (size_t)nk > max_cells) {
            for (auto* k : kids) delete k;
            out->push_back(q->id);
            continue;
        }
        count = count - 1 + (size_t)nk;
        for (int k = 0; k < 4; ++k) {
            if (!kids[k]) continue;
            if (cls[k] == kInside) { out->push_back(kids[k]->id); delete kids[k]; }
            else { owned.push_back(kids[k]); pq.push(kids[k]); }
        }
    }
    for (auto* q : owned) delete q;
    std::sort(out->begin(), out->end());
}

// Interior covering: cells wholly inside the polygon, largest first, at
// most max_cells, none below max_level.
void interior_covering(const Poly& P, uint32_t max_cells, int max_level, std::vector<uint64_t>* out) {
    std::vector<uint64_t> start;
    start_cells(P, &start);
    std::vector<QItem*> owned;
    std::priority_queue<QItem*, std::vector<QItem*>, QOrder> pq;
    std::vector<uint32_t> tmp;
    out->clear();
    for (uint64_t c : start) {
        const int cls = classify(P, c, nullptr, &tmp);
        if (cls == kInside) out->push_back(c);
        else if (cls == kBoundary) { owned.push_back(new QItem{c, tmp}); pq.push(owned.back()); }
    }
    while (!pq.empty() && out->size() < max_cells) {
        QItem* q = pq.top();
        pq.pop();
        if (cell_level(q->id) >= max_level) continue;
        for (int k = 0; k < 4 && out->size() < max_cells; ++k) {
            const uint64_t c = child_id(q->id, k);
            const int cls = classify(P, c, &q->edges, &tmp);
            if (cls == kInside) out->push_back(c);
            else if (cls == kBoundary) { owned.push_back(new QItem{c, tmp}); pq.push(owned.back()); }
        }
    }
    for (auto* q : owned) delete q;
    std::sort(out->begin(), out->end());
}

// ---------------------------------------------------------------------------
// super covering (§III-B, Listing "Build super covering")
// ---------------------------------------------------------------------------

using Refs = std::vector<uint32_t>;   // polygon_id << 1 | interior, ascending ids

void merge_ref(Refs* r, uint32_t ref) {
    const uint32_t pid = ref >> 1;
    auto it = std::lower_bound(r->begin(), r->end(), pid, [](uint32_t x, uint32_t p) { return (x >> 1) < p; });
    if (it != r->end() && (*it >> 1) == pid) {
        *it |= (ref & 1u);   // the same polygon as true and candidate: the interior (true) hit wins
        return;
    }
    r->insert(it, ref);
}

struct SuperCovering {
    std::map<uint64_t, Refs> cells;   // disjoint cells

    // the existing cell containing or equal to c, or end()
    std::map<uint64_t, Refs>::iterator containing(uint64_t c) {
        auto it = cells.upper_bound(c);
        if (it != cells.end() && cell_range_min(it->first) <= c) return it;
        if (it != cells.begin()) {
            auto p = std::prev(it);
            if (cell_range_max(p->first) >= c) return p;
        }
        return cells.end();
    }

    bool has_descendants(uint64_t c) {
        auto it = cells.lower_bound(cell_range_min(c));
        return it != cells.end() && it->first <= cell_range_max(c);
    }

    // c minus the existing cells inside it gets `ref`; the existing cells
    // inside c get `ref` merged in.
    void fill(uint64_t c, uint32_t ref) {
        auto ex = cells.find(c);
        if (ex != cells.end()) { merge_ref(&ex->second, ref); return; }
        if (!has_descendants(c)) { cells.emplace(c, Refs{ref}); return; }
        for (int k = 0; k < 4; ++k) fill(child_id(c, k), ref);
    }

    void insert(uint64_t c, uint32_t ref) {
        auto e = containing(c);
        if (e != cells.end()) {
            if (e->first == c) { merge_ref(&e->second, ref); return; }
            // conflict: existing ancestor c1 = e, descendant c2 = c; replace c1 by
            // c2 and the difference d (3 cells per level between them), all
            // carrying c1's references
            const uint64_t c1 = e->first;
            const Refs r1 = e->second;
            cells.erase(e);
            const int l1 = cell_level(c1), l2 = cell_level(c);
            for (int L = l1 + 1; L <= l2; ++L) {
                const uint64_t anc = cell_parent(c, L);
                const uint64_t par = cell_parent(c, L - 1);
                for (int k = 0; k < 4; ++k) {
                    const uint64_t sib = child_id(par, k);
                    if (sib != anc) cells.emplace(sib, r1);
                }
            }
            Refs r2 = r1;
            merge_ref(&r2, ref);
            cells.emplace(c, r2);
            return;
        }
        fill(c, ref);
    }
};

// ---------------------------------------------------------------------------
// refinement of candidate cells (approx precision and training)
// ---------------------------------------------------------------------------

struct CandRef {
    uint32_t poly;
    std::vector<uint32_t> edges;
};

struct OutCell {
    uint64_t id;
    Refs refs;
};

// Splits `id` into its children; each child keeps the true references and
// re-classifies the candidate ones.  Children with no reference are dropped
// (false hits).  Child candidates come with their edge lists.
void split_children(const std::vector<Poly>& polys, uint64_t id, const Refs& trues, const std::vector<CandRef>& cands,
                    std::vector<std::pair<OutCell, std::vector<CandRef>>>* out) {
    std::vector<uint32_t> tmp;
    for (int k = 0; k < 4; ++k) {
        const uint64_t c = child_id(id, k);
        OutCell oc{c, trues};
        std::vector<CandRef> cc;
        for (const CandRef& cr : cands) {
            const int cls = classify(polys[cr.poly], c, &cr.edges, &tmp);
            if (cls == kInside) merge_ref(&oc.refs, cr.poly << 1 | 1u);
            else if (cls == kBoundary) cc.push_back(CandRef{cr.poly, tmp});
        }
        if (oc.refs.empty() && cc.empty()) continue;
        out->push_back({std::move(oc), std::move(cc)});
    }
}

// Re-classifies a cell's candidate references against their polygons.
void reclassify(const std::vector<Poly>& polys, uint64_t id, const Refs& refs, Refs* trues, std::vector<CandRef>* cands) {
    std::vector<uint32_t> tmp;
    trues->clear();
    cands->clear();
    for (uint32_t r : refs) {
        if (r & 1u) { trues->push_back(r); continue; }
        const int cls = classify(polys[r >> 1], id, nullptr, &tmp);
        if (cls == kInside) merge_ref(trues, r | 1u);
        else if (cls == kBoundary) cands->push_back(CandRef{r >> 1, tmp});
    }
}

Refs with_cands(const Refs& trues, const std::vector<CandRef>& cands) {
    Refs r = trues;
    for (const CandRef& c : cands) merge_ref(&r, c.poly << 1);
    return r;
}

// Approximate mode: split candidate cells until diagonal + slack < eps.
void refine_approx(const std::vector<Poly>& polys, uint64_t id, const Refs& trues, const std::vector<CandRef>& cands,
                   double eps, std::vector<OutCell>* out) {
    if (cands.empty()) {
        if (!trues.empty()) out->push_back(OutCell{id, trues});
        return;
    }
    if (cell_level(id) >= kLevels || cell_diag_m(id) + kDiagSlack < eps) {
        out->push_back(OutCell{id, with_cands(trues, cands)});
        return;
    }
    std::vector<std::pair<OutCell, std::vector<CandRef>>> kids;
    split_children(polys, id, trues, cands, &kids);
    for (auto& k : kids) refine_approx(polys, k.first.id, k.first.refs, k.second, eps, out);
}

// ---------------------------------------------------------------------------
// trie sizing
// ---------------------------------------------------------------------------

struct FacePrefix {
    bool used = false;
    int P = 0;             // root prefix level (multiple of 4)
    uint64_t prefix = 0;   // top 2P key bits, right-aligned
};

void face_prefixes(const std::vector<uint64_t>& cells, FacePrefix fp[6]) {
    for (int f = 0; f < 6; ++f) fp[f] = FacePrefix();
    size_t a = 0;
    while (a < cells.size()) {
        const int f = (int)(cells[a] >> 61);
        size_t b = a;
        int min_level = kLevels;
        while (b < cells.size() && (int)(cells[b] >> 61) == f) {
            min_level = std::min(min_level, cell_level(cells[b]));
            ++b;
        }
        const uint64_t lo = cell_range_min(cells[a]) << 3, hi = cell_range_max(cells[b - 1]) << 3;
        const uint64_t x = lo ^ hi;
        const int common_bits = x ? __builtin_clzll(x) : 64;
        int P = std::min(common_bits / 2, min_level - 1);
        P = std::max(0, P / 4 * 4);
        fp[f].used = true;
        fp[f].P = P;
        fp[f].prefix = P ? lo >> (64 - 2 * P) : 0;
        a = b;
    }
}

inline int target_level(int L) { return (L + 3) / 4 * 4; }

// Node keys (aligned ancestor ids) a cell needs given the face root level P.
template <class F>
void for_node_keys(uint64_t cell, int P, F&& fn) {
    const int T = target_level(cell_level(cell));
    for (int A = P; A < T; A += 4) fn(A == 0 ? ((cell >> 61) << 61 | (1ull << 60)) : cell_parent(cell, A));
}

uint64_t count_nodes(const std::vector<uint64_t>& cells, const FacePrefix fp[6]) {
    std::unordered_set<uint64_t> keys;
    keys.reserve(cells.size());
    for (uint64_t c : cells) for_node_keys(c, fp[c >> 61].P, [&](uint64_t k) { keys.insert(k); });
    return keys.size();
}

// ---------------------------------------------------------------------------
// training (§III-D)
// ---------------------------------------------------------------------------

// Training from the training points' leaf cell ids (pid, kInvalidId for an
// invalid point): passes of hit counting on expensive cells (those with a
// candidate reference, below max_level) and splits in descending hit
// count, ties by cell id, until the node budget is spent or no expensive
// cell is hit.
void train_ids(const std::vector<Poly>& polys, std::vector<uint64_t>* cells, std::vector<Refs>* refs,
               const std::vector<uint64_t>& pid, uint64_t budget_bytes, int max_level, unsigned threads) {
    const uint64_t n_pts = pid.size();
    FacePrefix fp[6];
    face_prefixes(*cells, fp);
    std::unordered_set<uint64_t> node_keys;
    for (uint64_t c : *cells) for_node_keys(c, fp[c >> 61].P, [&](uint64_t k) { node_keys.insert(k); });
    const uint64_t node_bytes = (uint64_t)kNodeEntries * 8;
    bool budget_hit = false;
    for (int pass = 0; pass < 64 && !budget_hit; ++pass) {
        const size_t m = cells->size();
        std::vector<std::atomic<uint32_t>> hits(m);
        for (auto& h : hits) h.store(0, std::memory_order_relaxed);
        std::vector<uint8_t> expensive(m, 0);
        for (size_t k = 0; k < m; ++k) {
            if (cell_level((*cells)[k]) >= max_level) continue;
            for (uint32_t r : (*refs)[k])
                if (!(r & 1u)) { expensive[k] = 1; break; }
        }
        parallel_for(n_pts, threads, [&](size_t k, unsigned) {
            const uint64_t id = pid[k];
            if (id == kInvalidId) return;
            auto it = std::upper_bound(cells->begin(), cells->end(), id);
            size_t idx = (size_t)(it - cells->begin());
            if (it != cells->end() && cell_range_min(*it) <= id) {
            } else if (it != cells->begin() && cell_range_max(*(it - 1)) >= id) {
                idx -= 1;
            } else {
                return;
            }
            if (expensive[idx]) hits[idx].fetch_add(1, std::memory_order_relaxed);
        });
        std::vector<size_t> order;
        for (size_t k = 0; k < m; ++k)
            if (hits[k].load() > 0) order.push_back(k);
        if (order.empty()) break;
        std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            const uint32_t ha = hits[a].load(), hb = hits[b].load();
            if (ha != hb) return ha > hb;
            return (*cells)[a] < (*cells)[b];
        });
        std::vector<std::vector<OutCell>> repl(m);
        std::vector<uint8_t> replaced(m, 0);
        for (size_t k : order) {
            Refs trues;
            std::vector<CandRef> cands;
            reclassify(polys, (*cells)[k], (*refs)[k], &trues, &cands);
            std::vector<std::pair<OutCell, std::vector<CandRef>>> kids;
            if (!cands.empty()) split_children(polys, (*cells)[k], trues, cands, &kids);
            else kids.push_back({OutCell{(*cells)[k], trues}, {}});
            std::vector<uint64_t> new_keys;
            for (auto& kd : kids)
                for_node_keys(kd.first.id, fp[kd.first.id >> 61].P, [&](uint64_t key) {
                    if (!node_keys.count(key)) new_keys.push_back(key);
                });
            std::sort(new_keys.begin(), new_keys.end());
            new_keys.erase(std::unique(new_keys.begin(), new_keys.end()), new_keys.end());
            if ((node_keys.size() + new_keys.size()) * node_bytes > budget_bytes) { budget_hit = true; break; }
            for (uint64_t key : new_keys) node_keys.insert(key);
            for (auto& kd : kids) repl[k].push_back(OutCell{kd.first.id, with_cands(kd.first.refs, kd.second)});
            replaced[k] = 1;
        }
        std::vector<uint64_t> nc;
        std::vector<Refs> nr;
        nc.reserve(m + 3 * order.size());
        nr.reserve(m + 3 * order.size());
        for (size_t k = 0; k < m; ++k) {
            if (!replaced[k]) { nc.push_back((*cells)[k]); nr.push_back(std::move((*refs)[k])); continue; }
            for (auto& oc : repl[k]) { nc.push_back(oc.id); nr.push_back(std::move(oc.refs)); }
        }
        cells->swap(nc);
        refs->swap(nr);
    }
}

void train(const std::vector<Poly>& polys, std::vector<uint64_t>* cells, std::vector<Refs>* refs, const double* pts,
           uint64_t n_pts, uint64_t budget_bytes, int max_level, unsigned threads) {
    std::vector<uint64_t> pid(n_pts);
    parallel_for(n_pts, threads, [&](size_t k, unsigned) { pid[k] = point_cell_id(pts[2 * k], pts[2 * k + 1]); });
    train_ids(polys, cells, refs, pid, budget_bytes, max_level, threads);
}

// ---------------------------------------------------------------------------
// flattening (§III-C)
// ---------------------------------------------------------------------------

struct VecHash {
    size_t operator()(const std::vector<uint32_t>& v) const {
        uint64_t h = 1469598103934665603ull;
        for (uint32_t x : v) { h ^= x; h *= 1099511628211ull; }
        return (size_t)h;
    }
};

using LutMap = std::unordered_map<std::vector<uint32_t>, uint32_t, VecHash>;

// Encodes one reference list as [n_true, true ids..., n_cand, cand ids...]
// (§III-C "Lookup table"), stores it once, and returns its word offset.
bool lut_insert(const uint32_t* r, uint32_t nr, std::vector<uint32_t>* lut, LutMap* ids, uint32_t* off) {
    std::vector<uint32_t> enc;
    uint32_t nt = 0;
    for (uint32_t t = 0; t < nr; ++t) nt += r[t] & 1u;
    enc.push_back(nt);
    for (uint32_t t = 0; t < nr; ++t)
        if (r[t] & 1u) enc.push_back(r[t] >> 1);
    enc.push_back(nr - nt);
    for (uint32_t t = 0; t < nr; ++t)
        if (!(r[t] & 1u)) enc.push_back(r[t] >> 1);
    auto it = ids->find(enc);
    if (it != ids->end()) { *off = it->second; return true; }
    if (lut->size() > kPayloadMask) return false;
    *off = (uint32_t)lut->size();
    lut->insert(lut->end(), enc.begin(), enc.end());
    ids->emplace(std::move(enc), *off);
    return true;
}

int flatten(Index* idx, std::string* err) {
    idx->nodes.clear();
    idx->lut.clear();
    for (auto& f : idx->faces) f = FaceRoot{kNoRoot, 0, 0};
    FacePrefix fp[6];
    face_prefixes(idx->cells, fp);
    LutMap lut_ids;
    auto new_node = [&]() -> uint64_t {
        const uint64_t k = idx->nodes.size() / kNodeEntries;
        idx->nodes.resize(idx->nodes.size() + kNodeEntries, 0ull);
        return k;
    };
    uint32_t max_depth = 0, max_refs = 0, max_cand = 0, max_level = 0;
    uint64_t n_cand_cells = 0;
    for (int f = 0; f < 6; ++f)
        if (fp[f].used) idx->faces[f] = FaceRoot{(uint32_t)new_node(), (uint32_t)(2 * fp[f].P), fp[f].prefix};
    for (size_t k = 0; k < idx->cells.size(); ++k) {
        const uint64_t cell = idx->cells[k];
        const int f = (int)(cell >> 61);
        const int P = fp[f].P;
        const int L = cell_level(cell);
        const int T = target_level(L);
        const int depth = (T - P) / 4 - 1;
        uint64_t key = (cell_range_min(cell) << 3);
        if (P) key <<= 2 * P;
        uint64_t node = idx->faces[f].root;
        for (int d = 0; d < depth; ++d) {
            const uint32_t byte = (uint32_t)(key >> 56);
            key <<= 8;
            uint64_t& e = idx->nodes[node * kNodeEntries + byte];
            if (e == 0) {
                const uint64_t child = new_node();
                idx->nodes[node * kNodeEntries + byte] = child << kNodeShift;
                node = child;
            } else if ((e & kTagMask) != kTagPtr) {
                *err = "overlapping cells in the logical index";
                return AGJ_EINVAL;
            } else {
                node = e >> kNodeShift;
            }
        }
        // payload
        const uint32_t* r = idx->refs.data() + idx->ref_off[k];
        const uint32_t nr = (uint32_t)(idx->ref_off[k + 1] - idx->ref_off[k]);
        uint32_t nt = 0;
        for (uint32_t t = 0; t < nr; ++t) nt += r[t] & 1u;
        const uint32_t nc = nr - nt;
        max_refs = std::max(max_refs, nr);
        max_cand = std::max(max_cand, nc);
        if (nc) ++n_cand_cells;
        uint64_t entry;
        if (nr == 1) {
            entry = ((uint64_t)r[0] << 2) | kTagOne;
        } else if (nr == 2) {
            entry = ((uint64_t)r[1] << 33) | ((uint64_t)r[0] << 2) | kTagTwo;
        } else {
            uint32_t off;
            if (!lut_insert(r, nr, &idx->lut, &lut_ids, &off)) { *err = "lookup table too large"; return AGJ_EUNSUPPORTED; }
            entry = ((uint64_t)off << 2) | kTagLut;
        }
        const uint32_t cnt = 1u << (2 * (T - L));
        const uint32_t byte0 = (uint32_t)(key >> 56) & ~(cnt - 1u);
        for (uint32_t b = byte0; b < byte0 + cnt; ++b) {
            uint64_t& e = idx->nodes[node * kNodeEntries + b];
            if (e != 0) { *err = "overlapping cells in the logical index"; return AGJ_EINVAL; }
            e = entry;
        }
        max_depth = std::max(max_depth, (uint32_t)depth + 1);
        max_level = std::max(max_level, (uint32_t)L);
    }
    idx->stats.n_nodes = idx->nodes.size() / kNodeEntries;
    idx->stats.n_lut_words = idx->lut.size();
    idx->stats.max_refs = max_refs;
    idx->stats.max_cand_refs = max_cand;
    idx->stats.max_depth = max_depth;
    idx->stats.max_level = max_level;
    idx->stats.n_cand_cells = n_cand_cells;
    idx->stats.n_cells = idx->cells.size();
    return AGJ_OK;
}

}  // namespace

void lut_encode(const uint32_t* refs, const uint64_t* ref_off, uint64_t n_lists, std::vector<uint32_t>* words,
                std::vector<uint64_t>* offsets) {
    LutMap ids;
    words->clear();
    offsets->clear();
    for (uint64_t k = 0; k < n_lists; ++k) {
        uint32_t off = 0;
        lut_insert(refs + ref_off[k], (uint32_t)(ref_off[k + 1] - ref_off[k]), words, &ids, &off);
        offsets->push_back(off);
    }
}

void supercover(const uint64_t* cells, const uint32_t* refs, uint64_t n, std::vector<uint64_t>* out_cells,
                std::vector<uint64_t>* out_off, std::vector<uint32_t>* out_refs) {
    SuperCovering sc;
    for (uint64_t k = 0; k < n; ++k) sc.insert(cells[k], refs[k]);
    out_cells->clear();
    out_off->assign(1, 0);
    out_refs->clear();
    for (auto& kv : sc.cells) {
        out_cells->push_back(kv.first);
        out_refs->insert(out_refs->end(), kv.second.begin(), kv.second.end());
        out_off->push_back(out_refs->size());
    }
}

void poly_edges(const Index& X, uint32_t k, std::vector<uint32_t>* out) {
    out->clear();
    const uint32_t V = X.poly_off[k + 1] - X.poly_off[k];
    if (X.ring_off.size() != X.n_polys + 1 || X.ring_off[k + 1] == X.ring_off[k]) {
        for (uint32_t t = 0; t < V; ++t) out->push_back(t);
        return;
    }
    uint32_t start = 0;
    for (uint32_t q = X.ring_off[k]; q < X.ring_off[k + 1]; ++q) {
        const uint32_t end = X.ring_end[q];          // the closing duplicate is end - 1
        for (uint32_t t = start; t + 1 < end; ++t) out->push_back(t);
        start = end;
    }
}

int build_host(const agj_polygon* polys, uint32_t n_polys, const BuildParams& bp, Index* out, std::string* err) {
    const auto t0 = std::chrono::steady_clock::now();
    if (n_polys > 0 && !polys) { *err = "null polygon array"; return AGJ_EINVAL; }
    if (n_polys >= kMaxPolys) { *err = "too many polygons"; return AGJ_EUNSUPPORTED; }
    if (bp.mode == AGJ_APPROX && !(bp.precision_m > 0.0)) { *err = "precision must be > 0"; return AGJ_EINVAL; }
    const unsigned threads = bp.threads ? bp.threads : std::max(1u, std::thread::hardware_concurrency());
    Index& X = *out;
    X.mode = bp.mode;
    X.n_input_polys = n_polys;
    X.precision_m = bp.precision_m;
    // Validate the ring lists, then turn every polygon into pieces: one per
    // cube face it reaches, each the whole polygon in that face's gnomonic
    // (u,v) plane (its geodesic edges are straight there, and points on the
    // face are tested against it).  A polygon on one face is one piece with
    // the face coordinates of its vertices.  A polygon across faces must lie
    // within 15 degrees of its vertices' normalised mean c; it gets a piece on
    // each face whose axis is within 69.75 degrees of c (the faces its cap
    // can reach; every vertex is then in the face's open hemisphere) and
    // whose square its bbox meets.  Pieces are ordered by polygon, so piece
    // ids map to polygon ids monotonically (piece_poly).
    std::vector<uint32_t> piece_src;       // input polygon of each piece
    std::vector<int> piece_face;
    for (uint32_t k = 0; k < n_polys; ++k) {
        const agj_polygon& g = polys[k];
        if (g.n_vertices < 3 || !g.latlng) { *err = "polygon needs >= 3 vertices"; return AGJ_EINVAL; }
        if (g.n_rings >= 2) {
            if (!g.ring_ends) { *err = "polygon with holes needs ring ends"; return AGJ_EINVAL; }
            uint32_t prev = 0;
            for (uint32_t q = 0; q < g.n_rings; ++q) {
                if (g.ring_ends[q] < prev + 3 || g.ring_ends[q] > g.n_vertices) {
                    *err = "each ring needs >= 3 vertices and ring ends must ascend to n_vertices";
                    return AGJ_EINVAL;
                }
                prev = g.ring_ends[q];
            }
            if (prev != g.n_vertices) { *err = "the last ring end must be n_vertices"; return AGJ_EINVAL; }
        }
        int face = -1;
        bool one_face = true;
        double c[3] = {0.0, 0.0, 0.0};
        for (uint32_t t = 0; t < g.n_vertices; ++t) {
            const double lat = g.latlng[2 * t], lng = g.latlng[2 * t + 1];
            if (!point_valid(lat, lng)) { *err = "invalid polygon vertex"; return AGJ_EINVAL; }
            double u, v, xyz[3];
            const int f = face_uv(lat, lng, &u, &v);
            if (face >= 0 && f != face) one_face = false;
            face = f;
            latlng_xyz(lat, lng, xyz);
            c[0] += xyz[0]; c[1] += xyz[1]; c[2] += xyz[2];
        }
        if (one_face) {
            piece_src.push_back(k);
            piece_face.push_back(face);
            continue;
        }
        const double n = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int q = 0; q < 3; ++q) c[q] /= n;
        for (uint32_t t = 0; t < g.n_vertices; ++t) {
            double xyz[3];
            latlng_xyz(g.latlng[2 * t], g.latlng[2 * t + 1], xyz);
            if (!(xyz[0] * c[0] + xyz[1] * c[1] + xyz[2] * c[2] >= kCapCos)) {
                *err = "a polygon across cube faces must lie within 15 degrees of its vertices' mean";
                return AGJ_EUNSUPPORTED;
            }
        }
        for (int f = 0; f < 6; ++f) {
            const double axis = f < 3 ? c[f] : -c[f - 3];
            if (axis < kCapFaceCos) continue;
            double bb[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
            for (uint32_t t = 0; t < g.n_vertices; ++t) {
                double xyz[3], u, v;
                latlng_xyz(g.latlng[2 * t], g.latlng[2 * t + 1], xyz);
                if (!xyz_uv_on_face(f, xyz, &u, &v)) { *err = "projection outside the face's hemisphere"; return AGJ_EUNSUPPORTED; }
                bb[0] = std::min(bb[0], u); bb[1] = std::max(bb[1], u);
                bb[2] = std::min(bb[2], v); bb[3] = std::max(bb[3], v);
            }
            if (bb[1] < -1.0 || bb[0] > 1.0 || bb[3] < -1.0 || bb[2] > 1.0) continue;
            piece_src.push_back(k);
            piece_face.push_back(f);
        }
    }
    const uint32_t n_pieces = (uint32_t)piece_src.size();
    if (n_pieces >= kMaxPolys) { *err = "too many polygon pieces"; return AGJ_EUNSUPPORTED; }
    X.n_polys = n_pieces;
    X.piece_poly.clear();
    if (n_pieces != n_polys) X.piece_poly = piece_src;
    X.poly_off.assign(n_pieces + 1, 0);
    X.ring_off.assign(n_pieces + 1, 0);
    X.ring_end.clear();
    for (uint32_t k = 0; k < n_pieces; ++k) {
        const agj_polygon& g = polys[piece_src[k]];
        if (g.n_rings >= 2) {
            // rings stored explicitly closed: one more vertex per ring
            for (uint32_t q = 0; q < g.n_rings; ++q) X.ring_end.push_back(g.ring_ends[q] + q + 1);
            X.poly_off[k + 1] = X.poly_off[k] + g.n_vertices + g.n_rings;
        } else {
            X.poly_off[k + 1] = X.poly_off[k] + g.n_vertices;
        }
        X.ring_off[k + 1] = (uint32_t)X.ring_end.size();
    }
    X.poly_uv.assign(2ull * X.poly_off[n_pieces], 0.0);
    X.poly_bbox.assign(4ull * n_pieces, 0.0);
    X.poly_face.assign(n_pieces, (int8_t)-1);
    std::vector<Poly> P(n_pieces);
    std::vector<std::vector<uint32_t>> edges(n_pieces);
    for (uint32_t k = 0; k < n_pieces; ++k) {
        const agj_polygon& g = polys[piece_src[k]];
        const int face = piece_face[k];
        double bb[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
        uint32_t out = X.poly_off[k], ring = 0, ring_first = out;
        for (uint32_t t = 0; t < g.n_vertices; ++t) {
            double u, v, xyz[3];
            latlng_xyz(g.latlng[2 * t], g.latlng[2 * t + 1], xyz);
            xyz_uv_on_face(face, xyz, &u, &v);       // = face_uv's (u,v) for a vertex on this face
            X.poly_uv[2 * out] = u;
            X.poly_uv[2 * out + 1] = v;
            ++out;
            bb[0] = std::min(bb[0], u); bb[1] = std::max(bb[1], u);
            bb[2] = std::min(bb[2], v); bb[3] = std::max(bb[3], v);
            if (g.n_rings >= 2 && t + 1 == g.ring_ends[ring]) {     // close the ring explicitly
                X.poly_uv[2 * out] = X.poly_uv[2 * ring_first];
                X.poly_uv[2 * out + 1] = X.poly_uv[2 * ring_first + 1];
                ++out;
                ++ring;
                ring_first = out;
            }
        }
        X.poly_face[k] = (int8_t)face;
        std::memcpy(&X.poly_bbox[4 * k], bb, sizeof bb);
        P[k] = Poly{face, &X.poly_uv[2 * X.poly_off[k]], X.poly_off[k + 1] - X.poly_off[k], {bb[0], bb[1], bb[2], bb[3]}};
        if (g.n_rings >= 2) {
            poly_edges(X, k, &edges[k]);
            P[k].edges = edges[k].data();
            P[k].n_edges = (uint32_t)edges[k].size();
        }
    }
    n_polys = n_pieces;       // from here on the index's polygons are the pieces

    // per-polygon coverings and interior coverings
    std::vector<std::vector<uint64_t>> cov(n_polys), inter(n_polys);
    parallel_for(n_polys, threads, [&](size_t k, unsigned) {
        covering(P[k], bp.max_cover_cells, (int)bp.max_cover_level, &cov[k]);
        interior_covering(P[k], bp.max_interior_cells, (int)bp.max_interior_level, &inter[k]);
    });
    // super covering: all coverings (candidate refs), then all interiors (true refs)
    SuperCovering sc;
    for (uint32_t k = 0; k < n_polys; ++k)
        for (uint64_t c : cov[k]) sc.insert(c, k << 1);
    for (uint32_t k = 0; k < n_polys; ++k)
        for (uint64_t c : inter[k]) sc.insert(c, k << 1 | 1u);
    std::vector<uint64_t> cells;
    std::vector<Refs> refs;
    cells.reserve(sc.cells.size());
    refs.reserve(sc.cells.size());
    for (auto& kv : sc.cells) { cells.push_back(kv.first); refs.push_back(std::move(kv.second)); }
    sc.cells.clear();

    if (bp.mode == AGJ_APPROX) {
        std::vector<std::vector<OutCell>> outs(cells.size());
        parallel_for(cells.size(), threads, [&](size_t k, unsigned) {
            Refs trues;
            std::vector<CandRef> cands;
            bool has_cand = false;
            for (uint32_t r : refs[k]) has_cand |= !(r & 1u);
            if (!has_cand) { outs[k].push_back(OutCell{cells[k], refs[k]}); return; }
            reclassify(P, cells[k], refs[k], &trues, &cands);
            refine_approx(P, cells[k], trues, cands, bp.precision_m, &outs[k]);
        });
        std::vector<uint64_t> nc;
        std::vector<Refs> nr;
        for (auto& o : outs)
            for (auto& oc : o) { nc.push_back(oc.id); nr.push_back(std::move(oc.refs)); }
        std::vector<size_t> ord(nc.size());
        for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
        std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return nc[a] < nc[b]; });
        cells.clear();
        refs.clear();
        for (size_t k : ord) { cells.push_back(nc[k]); refs.push_back(std::move(nr[k])); }
    } else if (bp.train && bp.n_train) {
        FacePrefix fp[6];
        face_prefixes(cells, fp);
        const uint64_t untrained = count_nodes(cells, fp) * (uint64_t)kNodeEntries * 8;
        const uint64_t budget = bp.budget ? bp.budget : std::max<uint64_t>(4 * untrained, untrained + (16ull << 20));
        train(P, &cells, &refs, bp.train, bp.n_train, budget, (int)bp.max_train_level, threads);
    }

    X.cells = std::move(cells);
    X.ref_off.assign(X.cells.size() + 1, 0);
    for (size_t k = 0; k < refs.size(); ++k) X.ref_off[k + 1] = X.ref_off[k] + refs[k].size();
    X.refs.clear();
    X.refs.reserve(X.ref_off.back());
    for (auto& r : refs) X.refs.insert(X.refs.end(), r.begin(), r.end());

    const int rc = flatten(&X, err);
    if (rc != AGJ_OK) return rc;
    const uint64_t trie_bytes = X.nodes.size() * 8 + X.lut.size() * 4;
    if (bp.mode == AGJ_APPROX && bp.budget && trie_bytes > bp.budget) {
        *err = "approximate index exceeds the memory budget";
        return AGJ_EBUDGET;
    }
    if (bp.fast_ids) fit_fast_model(&X, threads);
    prepare_poly_local(&X, bp.pip_bands);
    X.stats.fast_ids = (uint32_t)X.model.enabled;
    X.stats.fast_err_cells = X.model.enabled ? (double)X.model.err : 0.0;
    X.stats.mode = (uint32_t)bp.mode;
    X.stats.n_polys = X.n_input_polys;
    X.stats.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return AGJ_OK;
}

int retrain(Index* X, const uint64_t* ids, uint64_t n_ids, uint64_t budget, uint32_t max_level, unsigned threads,
            std::string* err) {
    if (X->mode != AGJ_EXACT) { *err = "training refines exact-mode indexes"; return AGJ_EINVAL; }
    threads = threads ? threads : std::max(1u, std::thread::hardware_concurrency());
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<Poly> P(X->n_polys);
    std::vector<std::vector<uint32_t>> edges(X->n_polys);
    for (uint32_t k = 0; k < X->n_polys; ++k) {
        const double* bb = &X->poly_bbox[4 * k];
        P[k] = Poly{X->poly_face[k], &X->poly_uv[2 * X->poly_off[k]], X->poly_off[k + 1] - X->poly_off[k],
                    {bb[0], bb[1], bb[2], bb[3]}};
        if (X->ring_off.size() == X->n_polys + 1 && X->ring_off[k + 1] > X->ring_off[k]) {
            poly_edges(*X, k, &edges[k]);
            P[k].edges = edges[k].data();
            P[k].n_edges = (uint32_t)edges[k].size();
        }
    }
    std::vector<uint64_t> cells = X->cells;
    std::vector<Refs> refs(cells.size());
    for (size_t k = 0; k < cells.size(); ++k)
        refs[k].assign(X->refs.begin() + X->ref_off[k], X->refs.begin() + X->ref_off[k + 1]);
    if (!budget) {
        FacePrefix fp[6];
        face_prefixes(cells, fp);
        const uint64_t now = count_nodes(cells, fp) * (uint64_t)kNodeEntries * 8;
        budget = std::max<uint64_t>(4 * now, now + (16ull << 20));
    }
    train_ids(P, &cells, &refs, std::vector<uint64_t>(ids, ids + n_ids), budget, (int)(max_level ? max_level : 24),
              threads);
    X->cells = std::move(cells);
    X->ref_off.assign(X->cells.size() + 1, 0);
    for (size_t k = 0; k < refs.size(); ++k) X->ref_off[k + 1] = X->ref_off[k] + refs[k].size();
    X->refs.clear();
    X->refs.reserve(X->ref_off.back());
    for (auto& r : refs) X->refs.insert(X->refs.end(), r.begin(), r.end());
    const int rc = flatten(X, err);
    if (rc != AGJ_OK) return rc;
    if (X->model.enabled) fit_fast_model(X, threads);
    X->stats.fast_ids = (uint32_t)X->model.enabled;
    X->stats.fast_err_cells = X->model.enabled ? (double)X->model.err : 0.0;
    X->stats.build_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return AGJ_OK;
}

}  // namespace agj
