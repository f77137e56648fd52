// agj_model.cpp — fits the certified fast cell-id model of an index (the
// FastModel of agj_geom.cuh) on the host.
//
// Window.  The union of the index's cells is bounded by the (u,v) bbox of
// their rectangles on their face; its preimage's lat/lng bbox is taken from
// dense samples of the bbox boundary (lat and lng have no interior extrema on
// a face) and widened by 1e-6 degree plus 1e-4 of its extent.  A point outside
// the window therefore lies in no indexed cell and joins nothing.  The model
// is enabled only when all cells lie on one face, the window spans at most
// 1 degree from its centre each way, and every sample of the window lies on
// that face with |u|, |v| < 0.95 (far from face edges and the i/j clamp).
//
// Fit.  X = 2^30 s and Y = 2^30 t of the FP64 spec are fitted by least
// squares (Householder QR) with all monomials a^p b^q, p + q <= 5, of the
// offsets from the window centre normalised by powers of two (so that the
// normalisation is exact in floating point).
//
// The same fit and bound give an FP32 model of U = 2^30 u and V = 2^30 v
// (the polygon-test coordinates) for the refine step.
//
// Bound.  The device arithmetic is IEEE FP32 + int64 and is reproduced here
// bit for bit (model_ij in agj_geom.cuh), so the model's value at any sample
// is exactly what the GPU computes there.  The error |model - spec| is the sum
// of a smooth truncation term and rounding noise; it is sampled on a
// 1024 x 1024 grid of the window (spacing 1/512 of the normalised half-width)
// plus its edges and corners.  Between samples the smooth part can exceed its
// sampled maximum by at most a factor 1 / (1 - n^2 h) (Markov's inequality for
// the degree-n remainder, n <= 8, h = 1/512: < 1.15), and the rounding noise
// by its own analytic bound, a few units of 2^-24 of the magnitude of the
// terms; err = 2 x sampled maximum + 2^-20 level-30 cells covers both with
// room.  A model whose err exceeds 1/4 of a level-30 cell is not used.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "agj_geom.cuh"
#include "agj_index.h"

namespace agj {
namespace {

constexpr double kPi = 3.14159265358979323846;

void uv_latlng(int face, double u, double v, double* lat, double* lng) {
    double p[3];
    face_uv_to_xyz(face, u, v, p);
    *lat = std::atan2(p[2], std::sqrt(p[0] * p[0] + p[1] * p[1])) * (180.0 / kPi);
    *lng = std::atan2(p[1], p[0]) * (180.0 / kPi);
}

// Least squares by Householder QR: A (m x n, row major), b (m) -> x (n).
bool lstsq(std::vector<double> A, std::vector<double> b, int m, int n, std::vector<double>* x) {
    for (int k = 0; k < n; ++k) {
        double nrm = 0;
        for (int i = k; i < m; ++i) nrm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        nrm = std::sqrt(nrm);
        if (nrm == 0) return false;
        const double alpha = A[(size_t)k * n + k] > 0 ? -nrm : nrm;
        std::vector<double> v(m, 0.0);
        for (int i = k; i < m; ++i) v[i] = A[(size_t)i * n + k];
        v[k] -= alpha;
        double vn = 0;
        for (int i = k; i < m; ++i) vn += v[i] * v[i];
        if (vn == 0) continue;
        for (int j = k; j < n; ++j) {
            double d = 0;
            for (int i = k; i < m; ++i) d += v[i] * A[(size_t)i * n + j];
            d = 2 * d / vn;
            for (int i = k; i < m; ++i) A[(size_t)i * n + j] -= d * v[i];
        }
        double d = 0;
        for (int i = k; i < m; ++i) d += v[i] * b[i];
        d = 2 * d / vn;
        for (int i = k; i < m; ++i) b[i] -= d * v[i];
    }
    x->assign(n, 0.0);
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * (*x)[j];
        if (A[(size_t)k * n + k] == 0) return false;
        (*x)[k] = s / A[(size_t)k * n + k];
    }
    return true;
}

// Monomial order of the fit: (0,0), (1,0), (0,1), then the 18 higher terms in
// the layout of model_eval.
struct Mono {
    int p, q;
};

std::vector<Mono> monomials() {
    std::vector<Mono> m = {{0, 0}, {1, 0}, {0, 1}};
    for (int p = 2; p <= 5; ++p) m.push_back({p, 0});
    for (int p = 1; p <= 4; ++p) m.push_back({p, 1});
    for (int p = 0; p <= 3; ++p) m.push_back({p, 2});
    for (int p = 0; p <= 2; ++p) m.push_back({p, 3});
    for (int p = 0; p <= 1; ++p) m.push_back({p, 4});
    m.push_back({0, 5});
    return m;
}

void spec_xy(double lat, double lng, double* X, double* Y, int* face, double* u, double* v) {
    *face = face_uv(lat, lng, u, v);
    *X = uv_to_st(*u) * 1073741824.0;
    *Y = uv_to_st(*v) * 1073741824.0;
}

template <class F>
void par(size_t n, unsigned threads, F&& fn) {
    threads = std::max(1u, threads);
    std::vector<std::thread> th;
    std::atomic<size_t> next(0);
    for (unsigned t = 0; t < threads; ++t)
        th.emplace_back([&] {
            for (;;) {
                const size_t k = next.fetch_add(1);
                if (k >= n) break;
                fn(k);
            }
        });
    for (auto& x : th) x.join();
}

}  // namespace

void fit_fast_model(Index* idx, unsigned threads) {
    FastModel& M = idx->model;
    std::memset(&M, 0, sizeof M);
    if (idx->cells.empty()) return;
    const int face = (int)(idx->cells.front() >> 61);
    if ((int)(idx->cells.back() >> 61) != face) return;   // cells on more than one face
    // (u,v) bbox of the cells
    double ub[4] = {1e300, -1e300, 1e300, -1e300};
    for (uint64_t c : idx->cells) {
        const int L = cell_level(c);
        uint32_t o = (uint32_t)face & 1u, i = 0, j = 0;
        for (int l = 1; l <= L; ++l) {
            const uint32_t d = (uint32_t)((c >> (61 - 2 * l)) & 3ull);
            uint32_t ib = d >> 1, jb = (d >> 1) ^ (d & 1u);
            if (o & 2u) { ib ^= 1u; jb ^= 1u; }
            if (o & 1u) { const uint32_t t = ib; ib = jb; jb = t; }
            i = (i << 1) | ib;
            j = (j << 1) | jb;
            if (d == 0u) o ^= 1u;
            else if (d == 3u) o ^= 3u;
        }
        const double sc = std::ldexp(1.0, -L);
        ub[0] = std::min(ub[0], st_to_uv(i * sc));
        ub[1] = std::max(ub[1], st_to_uv((i + 1) * sc));
        ub[2] = std::min(ub[2], st_to_uv(j * sc));
        ub[3] = std::max(ub[3], st_to_uv((j + 1) * sc));
    }
    for (int k = 0; k < 4; ++k) ub[k] += (k & 1 ? 1e-9 : -1e-9);
    // lat/lng bbox of the (u,v) bbox boundary
    double lat_lo = 1e300, lat_hi = -1e300, lng_lo = 1e300, lng_hi = -1e300;
    const int S = 4096;
    for (int e = 0; e < 4; ++e)
        for (int k = 0; k <= S; ++k) {
            const double t = (double)k / S;
            double u, v;
            if (e == 0) { u = ub[0] + t * (ub[1] - ub[0]); v = ub[2]; }
            else if (e == 1) { u = ub[0] + t * (ub[1] - ub[0]); v = ub[3]; }
            else if (e == 2) { u = ub[0]; v = ub[2] + t * (ub[3] - ub[2]); }
            else { u = ub[1]; v = ub[2] + t * (ub[3] - ub[2]); }
            double la, lo;
            uv_latlng(face, u, v, &la, &lo);
            lat_lo = std::min(lat_lo, la); lat_hi = std::max(lat_hi, la);
            lng_lo = std::min(lng_lo, lo); lng_hi = std::max(lng_hi, lo);
        }
    const double mlat = 1e-6 + 1e-4 * (lat_hi - lat_lo), mlng = 1e-6 + 1e-4 * (lng_hi - lng_lo);
    lat_lo -= mlat; lat_hi += mlat; lng_lo -= mlng; lng_hi += mlng;
    if (!(lat_hi - lat_lo < 2.0 && lng_hi - lng_lo < 2.0)) return;
    if (lat_lo < -89.0 || lat_hi > 89.0 || lng_lo < -179.0 || lng_hi > 179.0) return;
    // centre on a 2^-20 degree grid; normalisation by powers of two
    const double lat_c = std::round(0.5 * (lat_lo + lat_hi) * 1048576.0) / 1048576.0;
    const double lng_c = std::round(0.5 * (lng_lo + lng_hi) * 1048576.0) / 1048576.0;
    const double ha = std::max(lat_hi - lat_c, lat_c - lat_lo), hb = std::max(lng_hi - lng_c, lng_c - lng_lo);
    const int ka = (int)std::ceil(std::log2(ha)), kb = (int)std::ceil(std::log2(hb));
    const double Ha = std::ldexp(1.0, ka), Hb = std::ldexp(1.0, kb);
    // the window must lie on this face, well inside it
    for (int a = 0; a <= 64; ++a)
        for (int b = 0; b <= 64; ++b) {
            double u, v;
            const int f = face_uv(lat_lo + (lat_hi - lat_lo) * a / 64.0, lng_lo + (lng_hi - lng_lo) * b / 64.0, &u, &v);
            if (f != face || std::fabs(u) > 0.95 || std::fabs(v) > 0.95) return;
        }
    // least-squares fit on a Chebyshev grid of the window
    const std::vector<Mono> mono = monomials();
    const int nm = (int)mono.size();
    const int G = 48;
    std::vector<double> A((size_t)G * G * nm), bx((size_t)G * G), by((size_t)G * G), bu((size_t)G * G),
        bv((size_t)G * G);
    double Xc, Yc, uc, vc;
    int fc;
    spec_xy(lat_c, lng_c, &Xc, &Yc, &fc, &uc, &vc);
    for (int ia = 0; ia < G; ++ia)
        for (int ib = 0; ib < G; ++ib) {
            const double al = std::cos(kPi * (ia + 0.5) / G) * ha / Ha;
            const double be = std::cos(kPi * (ib + 0.5) / G) * hb / Hb;
            double X, Y, u, v;
            int f;
            spec_xy(lat_c + al * Ha, lng_c + be * Hb, &X, &Y, &f, &u, &v);
            const size_t r = (size_t)ia * G + ib;
            for (int k = 0; k < nm; ++k) A[r * nm + k] = std::pow(al, mono[k].p) * std::pow(be, mono[k].q);
            bx[r] = X - Xc;
            by[r] = Y - Yc;
            bu[r] = (u - uc) * 1073741824.0;
            bv[r] = (v - vc) * 1073741824.0;
        }
    std::vector<double> cx, cy, cu, cv;
    if (!lstsq(A, bx, G * G, nm, &cx) || !lstsq(A, by, G * G, nm, &cy)) return;
    const bool have_uv = lstsq(A, bu, G * G, nm, &cu) && lstsq(A, bv, G * G, nm, &cv);
    FastModel F;
    std::memset(&F, 0, sizeof F);
    F.enabled = 1;
    F.face = face;
    // offsets: raw-bit differences when each coordinate's window lies in one
    // binade (same sign and exponent, at most 2^46 ulps from the centre), else
    // fixed point in units of 2^-47 degree
    auto same_binade = [](double lo, double hi, double c) {
        const int64_t bl = double_bits(lo), bh = double_bits(hi), bc = double_bits(c);
        if ((bl >> 52) != (bc >> 52) || (bh >> 52) != (bc >> 52)) return false;
        const int64_t d1 = bl > bc ? bl - bc : bc - bl, d2 = bh > bc ? bh - bc : bc - bh;
        return d1 < (1ll << 46) && d2 < (1ll << 46);
    };
    if (same_binade(lat_lo, lat_hi, lat_c) && same_binade(lng_lo, lng_hi, lng_c)) {
        F.path = 1;
        F.split = 23;
        const int64_t a0 = double_bits(lat_lo), a1 = double_bits(lat_hi);
        const int64_t b0 = double_bits(lng_lo), b1 = double_bits(lng_hi);
        F.wlat_lo = std::min(a0, a1); F.wlat_hi = std::max(a0, a1);
        F.wlng_lo = std::min(b0, b1); F.wlng_hi = std::max(b0, b1);
        F.lat0 = double_bits(lat_c);
        F.lng0 = double_bits(lng_c);
        const int ea = (int)((F.lat0 >> 52) & 0x7FF), eb = (int)((F.lng0 >> 52) & 0x7FF);
        const double sga = lat_c < 0 ? -1.0 : 1.0, sgb = lng_c < 0 ? -1.0 : 1.0;
        F.sa_hi = (float)(sga * std::ldexp(1.0, 23 + ea - 1075 - ka));
        F.sa_lo = (float)(sga * std::ldexp(1.0, ea - 1075 - ka));
        F.sb_hi = (float)(sgb * std::ldexp(1.0, 23 + eb - 1075 - kb));
        F.sb_lo = (float)(sgb * std::ldexp(1.0, eb - 1075 - kb));
    } else {
        F.path = 2;
        F.split = 24;
        F.wlat_lo = dkey_bits(double_bits(lat_lo));
        F.wlat_hi = dkey_bits(double_bits(lat_hi));
        F.wlng_lo = dkey_bits(double_bits(lng_lo));
        F.wlng_hi = dkey_bits(double_bits(lng_hi));
        F.lat0 = deg_fixed47(double_bits(lat_c));
        F.lng0 = deg_fixed47(double_bits(lng_c));
        F.sa_hi = (float)std::ldexp(1.0, 24 - 47 - ka);
        F.sa_lo = (float)std::ldexp(1.0, -47 - ka);
        F.sb_hi = (float)std::ldexp(1.0, 24 - 47 - kb);
        F.sb_lo = (float)std::ldexp(1.0, -47 - kb);
    }
    const double X0 = Xc + cx[0], Y0 = Yc + cy[0];
    F.n0x = (int32_t)std::floor(X0);
    F.n0y = (int32_t)std::floor(Y0);
    F.f0xy[0] = (float)(X0 - F.n0x);
    F.f0xy[1] = (float)(Y0 - F.n0y);
    // coefficient k of coordinate c (0: X or U, 1: Y or V) at [2 k + c]
    auto split = [](double c, float* hi, float* lo) {
        *hi = (float)c;
        *lo = (float)(c - (double)*hi);
    };
    split(cx[1], &F.xyl[0], &F.xyl[2]);
    split(cx[2], &F.xyl[4], &F.xyl[6]);
    split(cy[1], &F.xyl[1], &F.xyl[3]);
    split(cy[2], &F.xyl[5], &F.xyl[7]);
    for (int k = 0; k < kFastHiTerms; ++k) {
        F.xyh[2 * k] = (float)cx[3 + k];
        F.xyh[2 * k + 1] = (float)cy[3 + k];
    }
    if (have_uv) {
        const double U0 = uc * 1073741824.0 + cu[0], V0 = vc * 1073741824.0 + cv[0];
        F.n0u = (int32_t)std::floor(U0);
        F.n0v = (int32_t)std::floor(V0);
        F.f0uv[0] = (float)(U0 - F.n0u);
        F.f0uv[1] = (float)(V0 - F.n0v);
        split(cu[1], &F.uvl[0], &F.uvl[2]);
        split(cu[2], &F.uvl[4], &F.uvl[6]);
        split(cv[1], &F.uvl[1], &F.uvl[3]);
        split(cv[2], &F.uvl[5], &F.uvl[7]);
        for (int k = 0; k < kFastHiTerms; ++k) {
            F.uvh[2 * k] = (float)cu[3 + k];
            F.uvh[2 * k + 1] = (float)cv[3 + k];
        }
    }
    // sampled bound with the device-identical arithmetic: an (N+1) x (N+1)
    // grid including the window's edges and corners
    const int N = 1024;
    std::vector<double> worst(N + 1, 0.0), worst_base(N + 1, 0.0), worst_uv(N + 1, 0.0);
    std::vector<uint8_t> bad(N + 1, 0);
    par((size_t)N + 1, threads ? threads : std::thread::hardware_concurrency(), [&](size_t ia) {
        double w = 0, wb = 0, wu = 0;
        const double lat = ia == (size_t)N ? lat_hi : lat_lo + (lat_hi - lat_lo) * (double)ia / N;
        for (int ib = 0; ib <= N; ++ib) {
            const double lng = ib == N ? lng_hi : lng_lo + (lng_hi - lng_lo) * (double)ib / N;
            double u, v;
            face_uv(lat, lng, &u, &v);
            float ah, al, bh, bl;
            if (!model_offsets(F, double_bits(lat), double_bits(lng), &ah, &al, &bh, &bl)) { bad[ia] = 1; continue; }
            float xth, xtl, yth, ytl;
            model_eval_xy(F.xyl, F.xyh, F.f0xy, ah, al, bh, bl, &xth, &xtl, &yth, &ytl);
            const double dx = model_value(F.n0x, xth, xtl) - uv_to_st(u) * 1073741824.0;
            const double dy = model_value(F.n0y, yth, ytl) - uv_to_st(v) * 1073741824.0;
            w = std::max(w, std::max(std::fabs(dx), std::fabs(dy)));
            wb = std::max(wb, (double)std::max(std::fabs((xth - model_floor(xth)) + xtl), std::fabs((yth - model_floor(yth)) + ytl)));
            if (have_uv) {
                float uth, utl, vth, vtl;
                model_eval_xy(F.uvl, F.uvh, F.f0uv, ah, al, bh, bl, &uth, &utl, &vth, &vtl);
                // the model's real value n0 + th + tl (exact in double) against 2^30 (u, v)
                const double du = ((double)F.n0u + (double)uth + (double)utl) - u * 1073741824.0;
                const double dv = ((double)F.n0v + (double)vth + (double)vtl) - v * 1073741824.0;
                wu = std::max(wu, std::max(std::fabs(du), std::fabs(dv)));
            }
        }
        worst[ia] = w;
        worst_base[ia] = wb;
        worst_uv[ia] = wu;
    });
    double wmax = 0, bmax = 0, umax = 0;
    for (int k = 0; k <= N; ++k) {
        if (bad[k]) return;                                  // a window sample fell outside: inconsistent window
        wmax = std::max(wmax, worst[k]);
        bmax = std::max(bmax, worst_base[k]);
        umax = std::max(umax, worst_uv[k]);
    }
    if (have_uv) {
        const double eu = 2.0 * umax + std::ldexp(1.0, -16);
        if (eu < 0.25) {
            F.err_uv = (float)eu;
            if ((double)F.err_uv < eu) F.err_uv = std::nextafter(F.err_uv, 1.0f);
            F.uv_enabled = 1;
        }
    }
    // 2 x sampled maximum, plus rounding of base +- err (|base| < 64: ulp <= 2^-17)
    if (!(bmax < 64.0)) return;
    const double err = 2.0 * wmax + std::ldexp(1.0, -16);
    if (err > 0.25) return;                                  // more than 1/4 of a level-30 cell: not used
    F.err = (float)err;
    if ((double)F.err < err) F.err = std::nextafter(F.err, 1.0f);
    M = F;
}

// Horizontal bands of polygon k's certified test.  Band b covers local v in
// [bv0 + b h, bv0 + (b+1) h); it lists every edge whose v-range, widened by
// a margin M, meets that interval.  M exceeds the test's closeness bound D
// for any point that reaches the edge loop (D = (dp + dv) (1 + 1e-6), dp <=
// err_uv + (|u| + |v|) 2.4e-7 + 1e-5 with |u|, |v| within the bbox plus
// D), plus the rounding of the device's band index ((pv - bv0) / h in FP32:
// at most a unit of pv and a relative 2.4e-7 of the band count).  So every
// edge the all-edges loop could straddle, or whose vertex could come within
// D, is in the point's band: the banded test gives the same answer.
// A polygon with holes always gets a table (its edges are listed there, the
// device's all-edges loop assumes one ring) or, when none fits, no
// certified test at all (L->ok = 0: every candidate takes the FP64 test).
static void build_bands(Index* idx, uint32_t k, PolyLocal* L) {
    const uint32_t a = idx->poly_off[k], V = idx->poly_off[k + 1] - a;
    const bool holes = idx->ring_off.size() == idx->n_polys + 1 && idx->ring_off[k + 1] > idx->ring_off[k];
    if (!L->ok || !idx->model.uv_enabled) return;
    if (!holes && V < kBandMinVerts) return;
    const double lo = L->bv0, hi = L->bv1;
    if (!(hi > lo) || V > 65535) {
        if (holes) L->ok = 0;
        return;
    }
    const uint32_t nb = std::max<uint32_t>(1, std::min<uint32_t>(kBandMax, V / 4));
    const double h = (hi - lo) / nb;
    const double big = std::max(std::fabs((double)L->bu0), std::fabs((double)L->bu1)) +
                       std::max(std::fabs((double)L->bv0), std::fabs((double)L->bv1));
    const double M = 2.0 * ((double)idx->model.err_uv + (double)L->dv) + big * 5e-7 + 8.0 + h * 1e-3;
    std::vector<std::vector<uint16_t>> lists(nb);
    const F2* lv = idx->poly_luv.data() + a;
    std::vector<uint32_t> edges;
    poly_edges(*idx, k, &edges);
    for (const uint32_t e : edges) {
        const F2 A = lv[e], B = lv[e + 1 == V ? 0 : e + 1];
        const double ylo = std::min(A.y, B.y) - M, yhi = std::max(A.y, B.y) + M;
        const int64_t b0 = std::max<int64_t>(0, (int64_t)std::floor((ylo - lo) / h));
        const int64_t b1 = std::min<int64_t>(nb - 1, (int64_t)std::floor((yhi - lo) / h));
        for (int64_t b = b0; b <= b1; ++b) lists[b].push_back((uint16_t)e);
    }
    uint64_t total = nb + 1;
    for (auto& l : lists) total += l.size();
    if (total > kBandMaxWords) {                // too large to stage: test every edge
        if (holes) L->ok = 0;
        return;
    }
    L->band = (uint32_t)idx->poly_band.size();
    L->nb = nb;
    L->inv_h = (float)((double)nb / (hi - lo));
    L->band_len = (uint32_t)total;
    uint32_t off = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        idx->poly_band.push_back((uint16_t)off);
        off += (uint32_t)lists[b].size();
    }
    idx->poly_band.push_back((uint16_t)off);
    for (auto& l : lists) idx->poly_band.insert(idx->poly_band.end(), l.begin(), l.end());
}

void prepare_poly_local(Index* idx, bool bands) {
    const uint32_t P = idx->n_polys;
    idx->poly_local.assign(P, PolyLocal{});
    idx->poly_luv.assign(idx->poly_uv.size() / 2, F2{0.0f, 0.0f});
    idx->poly_band.clear();
    const double S = 1073741824.0;   // 2^30
    for (uint32_t k = 0; k < P; ++k) {
        const uint32_t a = idx->poly_off[k], b = idx->poly_off[k + 1];
        double u0 = 1e300, u1 = -1e300, v0 = 1e300, v1 = -1e300;
        for (uint32_t t = a; t < b; ++t) {
            u0 = std::min(u0, idx->poly_uv[2 * t] * S); u1 = std::max(u1, idx->poly_uv[2 * t] * S);
            v0 = std::min(v0, idx->poly_uv[2 * t + 1] * S); v1 = std::max(v1, idx->poly_uv[2 * t + 1] * S);
        }
        PolyLocal L{};      // no band table unless build_bands makes one
        L.ru = (int32_t)std::llround(0.5 * (u0 + u1));
        L.rv = (int32_t)std::llround(0.5 * (v0 + v1));
        // local coordinates must stay well inside 24-bit range
        L.ok = (u1 - L.ru < 8388608.0 && L.ru - u0 < 8388608.0 && v1 - L.rv < 8388608.0 && L.rv - v0 < 8388608.0) ? 1 : 0;
        double dv = 0;
        for (uint32_t t = a; t < b; ++t) {
            const double lu = idx->poly_uv[2 * t] * S - L.ru, lv = idx->poly_uv[2 * t + 1] * S - L.rv;   // exact
            const float fu = (float)lu, fv = (float)lv;
            idx->poly_luv[t] = F2{fu, fv};
            dv = std::max(dv, std::max(std::fabs((double)fu - lu), std::fabs((double)fv - lv)));
        }
        L.dv = (float)dv;
        if ((double)L.dv < dv) L.dv = std::nextafter(L.dv, 1.0f);
        L.bu0 = (float)(u0 - L.ru); L.bu1 = (float)(u1 - L.ru);
        L.bv0 = (float)(v0 - L.rv); L.bv1 = (float)(v1 - L.rv);
        // a polygon with holes needs its table whatever `bands` says
        if (bands || (idx->ring_off.size() == P + 1 && idx->ring_off[k + 1] > idx->ring_off[k]))
            build_bands(idx, k, &L);
        idx->poly_local[k] = L;
    }
}

}  // namespace agj
