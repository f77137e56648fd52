// agj_geom.cuh — point -> cell-id map and cell geometry, shared by the host
// index builder and the device kernels so both agree bit for bit.
//
// The paper uses S2 cell ids (§II "Google S2"): a point is projected onto a
// face of the unit cube, the face is subdivided as a quadtree and the cells
// are enumerated along a Hilbert curve; an id holds 3 face bits, up to 30
// bit pairs (one per level), a marker bit and a zero tail.  The paper does
// not fix the projection itself; this library fixes it as follows, using
// only IEEE + - * / sqrt floor round and comparisons in FP64 (host code is
// built with -ffp-contract=off, device code with -fmad=false, so nothing is
// fused):
//
//   sin/cos of degrees : q = round(d * fl(1/90)), r = d - 90 q (exact),
//                        x = r * fl(pi/180); odd Taylor series to x^17 and
//                        even to x^18 in Horner form; quadrant fix-up q mod 4
//   xyz                : (cos lat cos lng, cos lat sin lng, sin lat)
//   face               : axis of the largest |component| (ties to the lower
//                        axis), +3 if that component is negative
//   (u,v)              : ratios of the other components to the face one
//   (s,t)              : u >= 0 ? 0.5 sqrt(1+3u) : 1 - 0.5 sqrt(1-3u)
//   (i,j)              : clamp(floor(s 2^30), 0, 2^30-1)
//   position           : 30 Hilbert digits, MSB first; orientation bit 0
//                        swaps i/j, bit 1 inverts both; start = face & 1;
//                        canonical digits 0..3 = (0,0),(0,1),(1,1),(1,0);
//                        orientation ^= 1 after digit 0, ^= 3 after digit 3
//   id                 : face << 61 | position << 1 | 1
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define AGJ_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define AGJ_HD inline
#endif

#ifndef __CUDA_ARCH__
#include <cmath>
#endif

#ifdef __CUDA_ARCH__
#define AGJ_UNROLL _Pragma("unroll")
#else
#define AGJ_UNROLL
#endif

namespace agj {

constexpr int kLevels = 30;
constexpr uint64_t kInvalidId = 0;

AGJ_HD double geom_round(double x) {
#ifdef __CUDA_ARCH__
    return round(x);
#else
    return std::round(x);
#endif
}

AGJ_HD double geom_floor(double x) {
#ifdef __CUDA_ARCH__
    return floor(x);
#else
    return std::floor(x);
#endif
}

AGJ_HD double geom_sqrt(double x) {
#ifdef __CUDA_ARCH__
    return __dsqrt_rn(x);
#else
    return std::sqrt(x);
#endif
}

AGJ_HD double geom_fabs(double x) { return x < 0.0 ? -x : x; }

// sin and cos of an angle given in degrees.
AGJ_HD void sincos_deg(double d, double* s_out, double* c_out) {
    const double q = geom_round(d * (1.0 / 90.0));
    const double r = d - 90.0 * q;
    const double x = r * 0x1.1df46a2529d39p-6;      // fl(pi/180)
    const double z = x * x;
    // sin: x + (x z) h, h = -1/3! + z(1/5! + z(-1/7! + ... + z(1/17!)))
    double h = 1.0 / 355687428096000.0;             // 1/17!
    h = h * z - 1.0 / 1307674368000.0;              // 1/15!
    h = h * z + 1.0 / 6227020800.0;                 // 1/13!
    h = h * z - 1.0 / 39916800.0;                   // 1/11!
    h = h * z + 1.0 / 362880.0;                     // 1/9!
    h = h * z - 1.0 / 5040.0;                       // 1/7!
    h = h * z + 1.0 / 120.0;                        // 1/5!
    h = h * z - 1.0 / 6.0;                          // 1/3!
    const double sx = x + (x * z) * h;
    // cos: 1 + z g, g = -1/2! + z(1/4! + ... + z(-1/18!))
    double g = -1.0 / 6402373705728000.0;           // 1/18!
    g = g * z + 1.0 / 20922789888000.0;             // 1/16!
    g = g * z - 1.0 / 87178291200.0;                // 1/14!
    g = g * z + 1.0 / 479001600.0;                  // 1/12!
    g = g * z - 1.0 / 3628800.0;                    // 1/10!
    g = g * z + 1.0 / 40320.0;                      // 1/8!
    g = g * z - 1.0 / 720.0;                        // 1/6!
    g = g * z + 1.0 / 24.0;                         // 1/4!
    g = g * z - 1.0 / 2.0;                          // 1/2!
    const double cx = 1.0 + z * g;
    const int quadrant = (int)((long long)q & 3);
    if (quadrant == 0) { *s_out = sx;  *c_out = cx; }
    else if (quadrant == 1) { *s_out = cx;  *c_out = -sx; }
    else if (quadrant == 2) { *s_out = -sx; *c_out = -cx; }
    else { *s_out = -cx; *c_out = sx; }
}

AGJ_HD bool point_valid(double lat, double lng) {
    // NaN fails every comparison
    return geom_fabs(lat) <= 90.0 && geom_fabs(lng) <= 180.0;
}

// Face and (u,v) of a valid point.
AGJ_HD int face_uv(double lat, double lng, double* u, double* v) {
    double sp, cp, sl, cl;
    sincos_deg(lat, &sp, &cp);
    sincos_deg(lng, &sl, &cl);
    const double x = cp * cl, y = cp * sl, z = sp;
    const double ax = geom_fabs(x), ay = geom_fabs(y), az = geom_fabs(z);
    int face;
    if (ax >= ay && ax >= az) face = x < 0.0 ? 3 : 0;
    else if (ay >= az) face = y < 0.0 ? 4 : 1;
    else face = z < 0.0 ? 5 : 2;
    switch (face) {
        case 0: *u = y / x; *v = z / x; break;
        case 1: *u = -x / y; *v = z / y; break;
        case 2: *u = -x / z; *v = -y / z; break;
        case 3: *u = z / x; *v = y / x; break;
        case 4: *u = z / y; *v = -x / y; break;
        default: *u = -y / z; *v = -x / z; break;
    }
    return face;
}

// The unit vector of a point, as face_uv computes it.
AGJ_HD void latlng_xyz(double lat, double lng, double p[3]) {
    double sp, cp, sl, cl;
    sincos_deg(lat, &sp, &cp);
    sincos_deg(lng, &sl, &cl);
    p[0] = cp * cl;
    p[1] = cp * sl;
    p[2] = sp;
}

// (u,v) of a unit vector on the plane of `face` (the face's gnomonic
// coordinates, also beyond its square), with face_uv's expressions, so a
// point on that face gets exactly face_uv's (u,v).  False when the point is
// not in the face's open hemisphere.
AGJ_HD bool xyz_uv_on_face(int face, const double p[3], double* u, double* v) {
    const double x = p[0], y = p[1], z = p[2];
    switch (face) {
        case 0: if (!(x > 0.0)) return false; *u = y / x; *v = z / x; break;
        case 1: if (!(y > 0.0)) return false; *u = -x / y; *v = z / y; break;
        case 2: if (!(z > 0.0)) return false; *u = -x / z; *v = -y / z; break;
        case 3: if (!(x < 0.0)) return false; *u = z / x; *v = y / x; break;
        case 4: if (!(y < 0.0)) return false; *u = z / y; *v = -x / y; break;
        default: if (!(z < 0.0)) return false; *u = -y / z; *v = -x / z; break;
    }
    return true;
}

AGJ_HD double uv_to_st(double u) {
    if (u >= 0.0) return 0.5 * geom_sqrt(1.0 + 3.0 * u);
    return 1.0 - 0.5 * geom_sqrt(1.0 - 3.0 * u);
}

AGJ_HD double st_to_uv(double s) {
    if (s >= 0.5) return ((4.0 * s) * s - 1.0) / 3.0;
    const double w = 1.0 - s;
    return (1.0 - (4.0 * w) * w) / 3.0;
}

AGJ_HD uint32_t st_to_ij(double s) {
    const double k = geom_floor(s * 1073741824.0);
    if (k < 0.0) return 0u;
    if (k > 1073741823.0) return 1073741823u;
    return (uint32_t)k;
}

// One Hilbert step: quadrant bits (ib, jb) under orientation o -> digit,
// and the orientation of the child.
AGJ_HD uint32_t hilbert_digit(uint32_t ib, uint32_t jb, uint32_t* o) {
    if (*o & 1u) { const uint32_t t = ib; ib = jb; jb = t; }
    if (*o & 2u) { ib ^= 1u; jb ^= 1u; }
    const uint32_t digit = (ib << 1) | (ib ^ jb);
    if (digit == 0u) *o ^= 1u;
    else if (digit == 3u) *o ^= 3u;
    return digit;
}

// Position bits of levels 1..L (2L bits) of cell (i, j) given at level L.
AGJ_HD uint64_t hilbert_pos(int face, uint32_t i, uint32_t j, int L) {
    uint32_t o = (uint32_t)face & 1u;
    uint64_t pos = 0;
    for (int l = 1; l <= L; ++l) {
        const int sh = L - l;
        pos = (pos << 2) | hilbert_digit((i >> sh) & 1u, (j >> sh) & 1u, &o);
    }
    return pos;
}

// Cell id of cell (i, j) at level L of a face.
AGJ_HD uint64_t cell_id_from_ij(int face, uint32_t i, uint32_t j, int L) {
    const uint64_t pos = hilbert_pos(face, i, j, L);
    const int tail = 2 * (kLevels - L);
    return ((uint64_t)face << 61) | (pos << (tail + 1)) | (1ull << tail);
}

// Leaf cell id of a point; kInvalidId for an invalid point.
AGJ_HD uint64_t point_cell_id(double lat, double lng) {
    if (!point_valid(lat, lng)) return kInvalidId;
    double u, v;
    const int face = face_uv(lat, lng, &u, &v);
    return cell_id_from_ij(face, st_to_ij(uv_to_st(u)), st_to_ij(uv_to_st(v)), kLevels);
}

AGJ_HD int cell_level(uint64_t id) {
    int tz = 0;
    while (tz < 64 && ((id >> tz) & 1ull) == 0) ++tz;
    return kLevels - tz / 2;
}

AGJ_HD uint64_t cell_lsb(uint64_t id) { return id & (~id + 1ull); }
AGJ_HD uint64_t cell_range_min(uint64_t id) { return id - (cell_lsb(id) - 1ull); }
AGJ_HD uint64_t cell_range_max(uint64_t id) { return id + (cell_lsb(id) - 1ull); }

AGJ_HD uint64_t cell_parent(uint64_t id, int L) {
    const uint64_t lsb = 1ull << (2 * (kLevels - L));
    return (id & ~(2ull * lsb - 1ull)) | lsb;
}

// (u,v) of a point on a face given its (u,v) -> unit-sphere direction
// (not normalised).
AGJ_HD void face_uv_to_xyz(int face, double u, double v, double p[3]) {
    switch (face) {
        case 0: p[0] = 1.0; p[1] = u; p[2] = v; break;
        case 1: p[0] = -u; p[1] = 1.0; p[2] = v; break;
        case 2: p[0] = -u; p[1] = -v; p[2] = 1.0; break;
        case 3: p[0] = -1.0; p[1] = -v; p[2] = -u; break;
        case 4: p[0] = v; p[1] = -1.0; p[2] = -u; break;
        default: p[0] = v; p[1] = u; p[2] = -1.0; break;
    }
}

// ---------------------------------------------------------------------------
// Certified fast cell ids
// ---------------------------------------------------------------------------
// The FP64 id above costs ~150-200 FP64 instructions per point, and FP64 runs
// at a small fraction of the FP32 rate on this GPU.  For points inside an
// index's lat/lng window the library instead evaluates a local FP32 model of
// X = 2^30 s and Y = 2^30 t (degree-5 polynomials in the offsets from the
// window centre, first-order terms in double-float) together with a bound
// err on |model - spec| that the host derives when it fits the model.  The
// spec's i = floor(X) then lies in [floor(X - err), floor(X + err)]; the
// leading levels on which both ends agree are exactly the spec's, so the
// prefix of the id up to that level is bit-exact.  A walk that needs a
// deeper level than certified recomputes the FP64 id.
//
// All arithmetic here is IEEE FP32 / integer with explicit fmaf, so host and
// device produce identical values (host code -ffp-contract=off, device code
// -fmad=false); the host evaluates the very same function to bound the error.

constexpr int kFastHiTerms = 18;   // coefficients of degrees 2..5

// The two coordinates' coefficients are interleaved (X, Y), (X, Y), ... so
// that the device evaluates both as one pair of FP32 lanes (model_eval_xy).
struct FastModel {
    int32_t enabled;
    int32_t face;
    int32_t path;                   // 1: each coordinate in one binade (raw-bit offsets); 2: general
    int32_t n0x, n0y;               // integer parts of the constant terms (level-30 cells)
    float err;                      // bound on |model - spec| incl. rounding allowances (cells)
    alignas(8) float f0xy[2];       // fractional parts of the constant terms (X, Y)
    int64_t wlat_lo, wlat_hi, wlng_lo, wlng_hi;   // window: path 1 raw bits, path 2 order keys
    int64_t lat0, lng0;             // centre: path 1 raw bits, path 2 units of 2^-47 degree
    int32_t split;                  // bits in the low part of an offset (23 path 1, 24 path 2)
    float sa_hi, sa_lo, sb_hi, sb_lo;   // scales of the offsets' two parts (powers of two)
    alignas(8) float xyl[8];        // first order: c10 hi, c10 lo, c01 hi, c01 lo, each (X, Y)
    alignas(8) float xyh[2 * kFastHiTerms];   // degrees 2..5 (layout in model_eval), each (X, Y)
    // the same kind of model for U = 2^30 u and V = 2^30 v (the refine step)
    int32_t uv_enabled;
    int32_t n0u, n0v;
    float err_uv;                   // bound on |model - 2^30 (u,v)|, same units
    alignas(8) float f0uv[2];
    alignas(8) float uvl[8];
    alignas(8) float uvh[2 * kFastHiTerms];
};

AGJ_HD int64_t double_bits(double x) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    int64_t b;
    __builtin_memcpy(&b, &x, 8);
    return b;
#endif
}

AGJ_HD int32_t float_bits(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_int(x);
#else
    int32_t b;
    __builtin_memcpy(&b, &x, 4);
    return b;
#endif
}

// Order-preserving integer key of a double (sign-magnitude to two's
// complement; -0.0 and +0.0 share a key; NaNs fall outside every finite range).
AGJ_HD int64_t dkey_bits(int64_t b) { return b < 0 ? -(b & 0x7FFFFFFFFFFFFFFFll) : b; }

// x (given by its bits, |x| < 256) in units of 2^-47, truncated toward zero.
AGJ_HD int64_t deg_fixed47(int64_t b) {
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) return 0;
    const int64_t m = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = e - 1028;
    const int64_t f = sh >= 0 ? (m << sh) : (sh > -63 ? (m >> -sh) : 0);
    return b < 0 ? -f : f;
}

AGJ_HD float model_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

AGJ_HD float model_floor(float x) {
#ifdef __CUDA_ARCH__
    return floorf(x);
#else
    return std::floor(x);
#endif
}

// Error-free sum: s + e == a + b exactly (Knuth).
AGJ_HD void two_sum(float a, float b, float* s, float* e) {
    const float x = a + b;
    const float bv = x - a;
    const float av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

// Offsets of a point from the window centre, normalised and split into two
// floats whose exact sum is the offset.  Returns false outside the window.
AGJ_HD bool model_offsets(const FastModel& M, int64_t blat, int64_t blng, float* ah, float* al, float* bh, float* bl) {
    int64_t da, db;
    if (M.path == 1) {
        // every lat (lng) of the window shares sign and exponent: raw bits are
        // ordered like the values and their difference counts ulps
        if (blat < M.wlat_lo || blat > M.wlat_hi || blng < M.wlng_lo || blng > M.wlng_hi) return false;
        da = blat - M.lat0;
        db = blng - M.lng0;
    } else {
        const int64_t klat = dkey_bits(blat), klng = dkey_bits(blng);
        if (klat < M.wlat_lo || klat > M.wlat_hi || klng < M.wlng_lo || klng > M.wlng_hi) return false;
        da = deg_fixed47(blat) - M.lat0;
        db = deg_fixed47(blng) - M.lng0;
    }
    const int64_t mask = (1ll << M.split) - 1;
    *ah = (float)(int32_t)(da >> M.split) * M.sa_hi;
    *al = (float)(int32_t)(da & mask) * M.sa_lo;
    *bh = (float)(int32_t)(db >> M.split) * M.sb_hi;
    *bl = (float)(int32_t)(db & mask) * M.sb_lo;
    return true;
}

// Model value minus its integer constant, as th + tl (floats; th carries the
// large first-order and polynomial terms, tl the small remainder and the
// constant's fraction f0).  Coefficient k of one coordinate is L[2k] (first
// order) or H[2k] (higher terms; the other coordinate's sit between).
// H: b^0: a^2..a^5 (h0..h3); b^1: a^1..a^4 (h4..h7); b^2: a^0..a^3
// (h8..h11); b^3: a^0..a^2 (h12..h14); b^4: a^0, a^1 (h15, h16); b^5: h17.
AGJ_HD void model_eval(const float* L, const float* H, float f0, float ah, float al, float bh, float bl, float* th,
                       float* tl) {
    const float p1 = L[0] * ah;
    const float e1 = model_fma(L[0], ah, -p1);
    const float p2 = L[4] * bh;
    const float e2 = model_fma(L[4], bh, -p2);
    float corr = e1 + e2;
    corr = model_fma(L[0], al, corr);
    corr = model_fma(L[2], ah, corr);
    corr = model_fma(L[4], bl, corr);
    corr = model_fma(L[6], bh, corr);
    const float a = ah + al, b = bh + bl;
    const float q0 = (a * a) * model_fma(a, model_fma(a, model_fma(a, H[6], H[4]), H[2]), H[0]);
    const float q1 = a * model_fma(a, model_fma(a, model_fma(a, H[14], H[12]), H[10]), H[8]);
    const float q2 = model_fma(a, model_fma(a, model_fma(a, H[22], H[20]), H[18]), H[16]);
    const float q3 = model_fma(a, model_fma(a, H[28], H[26]), H[24]);
    const float q4 = model_fma(a, H[32], H[30]);
    float t = model_fma(b, H[34], q4);
    t = model_fma(b, t, q3);
    t = model_fma(b, t, q2);
    t = model_fma(b, t, q1);
    const float poly = model_fma(b, t, q0);
    float s1, r1, s2, r2;
    two_sum(p1, p2, &s1, &r1);
    two_sum(s1, poly, &s2, &r2);
    *th = s2;
    *tl = ((r1 + r2) + corr) + f0;
}

#ifdef __CUDA_ARCH__
// Paired FP32 lanes (fma/mul/add/sub .rn.f32x2: two independent
// round-to-nearest operations), for evaluating the two coordinates at once.
typedef unsigned long long f32x2_t;
__device__ __forceinline__ f32x2_t f2_pair(float x, float y) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void f2_split(f32x2_t v, float* x, float* y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(*x), "=f"(*y) : "l"(v));
}
__device__ __forceinline__ f32x2_t f2_fma(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2_t f2_mul(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_add(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_sub(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
#endif

// model_eval of both coordinates (interleaved coefficients L, H, f0): on the
// device as paired FP32 lanes with model_eval's operation order, so each
// lane's result equals model_eval's; on the host twice in turn.
AGJ_HD void model_eval_xy(const float* L, const float* H, const float* f0, float ah, float al, float bh, float bl,
                          float* xth, float* xtl, float* yth, float* ytl) {
#ifdef __CUDA_ARCH__
    const f32x2_t* Lp = reinterpret_cast<const f32x2_t*>(L);
    const f32x2_t* Hp = reinterpret_cast<const f32x2_t*>(H);
    const f32x2_t AH = f2_pair(ah, ah), AL = f2_pair(al, al), BH = f2_pair(bh, bh), BL = f2_pair(bl, bl);
    const f32x2_t NEG = f2_pair(-1.0f, -1.0f);
    const f32x2_t p1 = f2_mul(Lp[0], AH);
    const f32x2_t e1 = f2_fma(Lp[0], AH, f2_mul(p1, NEG));
    const f32x2_t p2 = f2_mul(Lp[2], BH);
    const f32x2_t e2 = f2_fma(Lp[2], BH, f2_mul(p2, NEG));
    f32x2_t corr = f2_add(e1, e2);
    corr = f2_fma(Lp[0], AL, corr);
    corr = f2_fma(Lp[1], AH, corr);
    corr = f2_fma(Lp[2], BL, corr);
    corr = f2_fma(Lp[3], BH, corr);
    const float a = ah + al, b = bh + bl;
    const f32x2_t A = f2_pair(a, a), B = f2_pair(b, b), AA = f2_pair(a * a, a * a);
    const f32x2_t q0 = f2_mul(AA, f2_fma(A, f2_fma(A, f2_fma(A, Hp[3], Hp[2]), Hp[1]), Hp[0]));
    const f32x2_t q1 = f2_mul(A, f2_fma(A, f2_fma(A, f2_fma(A, Hp[7], Hp[6]), Hp[5]), Hp[4]));
    const f32x2_t q2 = f2_fma(A, f2_fma(A, f2_fma(A, Hp[11], Hp[10]), Hp[9]), Hp[8]);
    const f32x2_t q3 = f2_fma(A, f2_fma(A, Hp[14], Hp[13]), Hp[12]);
    const f32x2_t q4 = f2_fma(A, Hp[16], Hp[15]);
    f32x2_t t = f2_fma(B, Hp[17], q4);
    t = f2_fma(B, t, q3);
    t = f2_fma(B, t, q2);
    t = f2_fma(B, t, q1);
    const f32x2_t poly = f2_fma(B, t, q0);
    // the two error-free sums of model_eval, lane by lane
    const f32x2_t s1 = f2_add(p1, p2);
    const f32x2_t bv1 = f2_sub(s1, p1);
    const f32x2_t av1 = f2_sub(s1, bv1);
    const f32x2_t r1 = f2_add(f2_sub(p1, av1), f2_sub(p2, bv1));
    const f32x2_t s2 = f2_add(s1, poly);
    const f32x2_t bv2 = f2_sub(s2, s1);
    const f32x2_t av2 = f2_sub(s2, bv2);
    const f32x2_t r2 = f2_add(f2_sub(s1, av2), f2_sub(poly, bv2));
    const f32x2_t tl = f2_add(f2_add(f2_add(r1, r2), corr), *reinterpret_cast<const f32x2_t*>(f0));
    f2_split(s2, xth, yth);
    f2_split(tl, xtl, ytl);
#else
    model_eval(L, H, f0[0], ah, al, bh, bl, xth, xtl);
    model_eval(L + 1, H + 1, f0[1], ah, al, bh, bl, yth, ytl);
#endif
}

// floor(n0 + th + tl - err) and floor(n0 + th + tl + err) for small |tl|
// (the floor of th is exact, so only the small remainder is rounded).
AGJ_HD void model_cells(int32_t n0, float th, float tl, float err, int32_t* lo, int32_t* hi) {
    const float k = model_floor(th);
    const float base = (th - k) + tl;
    const int32_t c = n0 + (int32_t)k;
    *lo = c + (int32_t)model_floor(base - err);
    *hi = c + (int32_t)model_floor(base + err);
}

// The model's value n0 + th + tl as a double (host-side bound checks).
AGJ_HD double model_value(int32_t n0, float th, float tl) {
    const float k = model_floor(th);
    const float base = (th - k) + tl;
    return (double)n0 + (double)k + (double)base;
}

AGJ_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// Fast certified (i, j) of a point.  Returns 0 when the point lies outside
// the model window (no indexed cell can hold it: the window contains every
// indexed cell), 1 with *lc = number of leading levels certified (0..30),
// i and j set from the lower end of the error interval.
AGJ_HD int model_ij(const FastModel& M, double lat, double lng, uint32_t* i, uint32_t* j, int* lc) {
    float ah, al, bh, bl;
    if (!model_offsets(M, double_bits(lat), double_bits(lng), &ah, &al, &bh, &bl)) return 0;
    float xth, xtl, yth, ytl;
    model_eval_xy(M.xyl, M.xyh, M.f0xy, ah, al, bh, bl, &xth, &xtl, &yth, &ytl);
    int32_t ilo, ihi, jlo, jhi;
    model_cells(M.n0x, xth, xtl, M.err, &ilo, &ihi);
    model_cells(M.n0y, yth, ytl, M.err, &jlo, &jhi);
    if (ilo < 0 || jlo < 0 || ihi > 1073741823 || jhi > 1073741823) {
        *i = 0; *j = 0; *lc = 0;
        return 1;
    }
    const int li = clz32((uint32_t)(ilo ^ ihi)) - 2, lj = clz32((uint32_t)(jlo ^ jhi)) - 2;
    *i = (uint32_t)ilo;
    *j = (uint32_t)jlo;
    *lc = li < lj ? li : lj;
    return 1;
}

// Hilbert table for 4 levels at a time: index (o << 8) | (i4 << 4) | j4,
// value (8 position bits << 2) | next orientation.
struct HilbertLut {
    uint16_t v[1024];
};

constexpr uint32_t hilbert_digit_c(uint32_t ib, uint32_t jb, uint32_t& o) {
    if (o & 1u) { const uint32_t t = ib; ib = jb; jb = t; }
    if (o & 2u) { ib ^= 1u; jb ^= 1u; }
    const uint32_t d = (ib << 1) | (ib ^ jb);
    if (d == 0u) o ^= 1u;
    else if (d == 3u) o ^= 3u;
    return d;
}

constexpr HilbertLut make_hilbert_lut() {
    HilbertLut L{};
    for (uint32_t idx = 0; idx < 1024; ++idx) {
        uint32_t o = idx >> 8, pos = 0;
        for (int l = 0; l < 4; ++l) pos = (pos << 2) | hilbert_digit_c((idx >> (7 - l)) & 1u, (idx >> (3 - l)) & 1u, o);
        L.v[idx] = (uint16_t)((pos << 2) | o);
    }
    return L;
}

AGJ_HD uint16_t hilbert_lut_entry(uint32_t idx) {
    uint32_t o = idx >> 8, pos = 0;
    for (int l = 0; l < 4; ++l) {
        const uint32_t ib = (idx >> (7 - l)) & 1u, jb = (idx >> (3 - l)) & 1u;
        pos = (pos << 2) | hilbert_digit(ib, jb, &o);
    }
    return (uint16_t)((pos << 2) | o);
}

// The leaf id's key bytes (the id shifted left by the 3 face bits): byte b
// holds the Hilbert digits of levels 4b+1 .. 4b+4, one table lookup each.
// Levels 31-32 of the last byte are zero padding (the id has its marker and
// zero tail there); the trie fills every combination of those bits for the
// few cells that deep, so the walk reads the same entry either way.
AGJ_HD uint64_t key_bytes_lut(const uint16_t* lut, int face, uint32_t i, uint32_t j) {
    const uint32_t i32 = i << 2, j32 = j << 2;
    uint32_t o = (uint32_t)face & 1u, hi = 0, lo = 0;
    AGJ_UNROLL
    for (int s = 0; s < 4; ++s) {
        const uint32_t e = lut[(o << 8) | (((i32 >> (28 - 4 * s)) & 15u) << 4) | ((j32 >> (28 - 4 * s)) & 15u)];
        hi = (hi << 8) | (e >> 2);
        o = e & 3u;
    }
    AGJ_UNROLL
    for (int s = 4; s < 8; ++s) {
        const uint32_t e = lut[(o << 8) | (((i32 >> (28 - 4 * s)) & 15u) << 4) | ((j32 >> (28 - 4 * s)) & 15u)];
        lo = (lo << 8) | (e >> 2);
        o = e & 3u;
    }
    return ((uint64_t)hi << 32) | lo;
}

// Leaf cell id from level-30 (i, j) with the 4-level table (same value as
// cell_id_from_ij(face, i, j, 30)).
AGJ_HD uint64_t cell_id_lut(const uint16_t* lut, int face, uint32_t i, uint32_t j) {
    const uint64_t key = key_bytes_lut(lut, face, i, j);
    return ((uint64_t)face << 61) | ((key >> 4) << 1) | 1ull;
}

// ---------------------------------------------------------------------------
// Certified ST_Covers in FP32 (the refine step)
// ---------------------------------------------------------------------------
// Coordinates are 2^30 (u, v) measured from a per-polygon integer reference
// point, held in FP32: a vertex's local coordinates carry a rounding error of
// at most PolyLocal::dv, a point's (from the U/V model) at most dp.  The ring
// rule of the spec is decided from them only where the decision is certain:
// every vertex v-comparison with the point must be farther apart than the
// summed errors, and on every edge that straddles the point the orientation
// must exceed its forward error bound (input errors times the other factors,
// plus FP32 rounding of the products and the difference).  Then the spec's
// FP64 orientation has the same sign and is not zero, so the crossing count
// and the "on an edge" outcome are the spec's.  Anything closer returns -1
// and the caller recomputes the point's (u, v) and the test in FP64.

struct F2 {
    float x, y;
};

struct PolyLocal {
    int32_t ru, rv;                 // reference point, units of 2^-30 in (u, v)
    float dv;                       // bound on the rounding of any local vertex coordinate
    float bu0, bu1, bv0, bv1;       // local bbox (rounded values of the exact bbox)
    int32_t ok;                     // 0: polygon too large for 24-bit local coordinates
    // horizontal bands over the bbox: band b (v in [bv0 + b h, bv0 + (b+1) h))
    // lists every edge whose v-range comes within a margin of it, so a point
    // tests only its band's edges (0 bands: every edge)
    uint32_t band;                  // offset of the band table in the index's band array (uint16 words)
    uint32_t nb;                    // bands
    float inv_h;                    // 1 / h
    uint32_t band_len;              // words of the table: nb + 1 edge offsets, then the edge indices
};

AGJ_HD float fabs_f(float x) { return x < 0.0f ? -x : x; }

// 1 covered, 0 not covered, -1 undecided.  verts: the ring's local
// coordinates (implicitly closed).
// One edge (A, B) of the certified crossing test; returns false when the
// point is too close to decide (a vertex within D in v, or the orientation
// within its error bound), else toggles *inside on a crossing.
AGJ_HD bool certified_edge(F2 A, F2 B, float dA, float dB, float pu, float ev, float ep, int* inside) {
    if ((dA > 0.0f) != (dB > 0.0f)) {
        const float d1 = B.x - A.x, d3 = B.y - A.y, d4 = pu - A.x;
        const float t1 = d1 * dA, t2 = d3 * d4;
        const float o = t1 - t2;
        const float e1 = ev + fabs_f(d1) * 6.0e-8f, e3 = ev + fabs_f(d3) * 6.0e-8f;
        const float e2 = ep + fabs_f(dA) * 6.0e-8f, e4 = ep + fabs_f(d4) * 6.0e-8f;
        const float bound = (fabs_f(d1) * e2 + fabs_f(dA) * e1 + e1 * e2 + fabs_f(d3) * e4 + fabs_f(d4) * e3 +
                             e3 * e4 + (fabs_f(t1) + fabs_f(t2)) * 2.4e-7f) * 1.0001f;
        if (fabs_f(o) <= bound) return false;
        // upward edge (a.v < p.v < b.v) crosses when o > 0, downward when o < 0
        if ((dA > 0.0f) == (o > 0.0f)) *inside ^= 1;
    }
    return true;
}

// Certified ST_Covers in FP32 local coordinates: 1 covered, 0 not, -1
// undecided (the caller recomputes in FP64).  With a band table (bands !=
// null, P.nb > 0) only the point's band's edges are tested: every edge that
// can straddle the point's v or bring a vertex within D of it is listed
// there, so the answer is the same as over all edges.
AGJ_HD int covers_certified(const F2* verts, uint32_t nv, const PolyLocal& P, const uint16_t* bands, float pu,
                            float pv, float dp) {
    const float D = (dp + P.dv) * 1.000001f;
    if (pu < P.bu0 - D || pu > P.bu1 + D || pv < P.bv0 - D || pv > P.bv1 + D) return 0;
    if (!(pu > P.bu0 + D && pu < P.bu1 - D && pv > P.bv0 + D && pv < P.bv1 - D)) return -1;
    const float ev = 2.0f * P.dv, ep = dp + P.dv;
    int inside = 0;
    if (bands && P.nb) {
        int b = (int)((pv - P.bv0) * P.inv_h);     // pv > bv0 here: truncation is floor
        b = b < 0 ? 0 : (b >= (int)P.nb ? (int)P.nb - 1 : b);
        const uint16_t* E = bands + P.nb + 1;
        for (uint32_t t = bands[b]; t < bands[b + 1]; ++t) {
            const uint32_t k = E[t];
            const F2 A = verts[k], B = verts[k + 1 == nv ? 0 : k + 1];
            const float dA = pv - A.y, dB = pv - B.y;
            if (fabs_f(dA) <= D || fabs_f(dB) <= D) return -1;
            if (!certified_edge(A, B, dA, dB, pu, ev, ep, &inside)) return -1;
        }
        return inside;
    }
    F2 A = verts[0];
    float dA = pv - A.y;
    if (fabs_f(dA) <= D) return -1;
    for (uint32_t k = 0; k < nv; ++k) {
        const F2 B = verts[k + 1 == nv ? 0 : k + 1];
        const float dB = pv - B.y;
        if (fabs_f(dB) <= D) return -1;
        if (!certified_edge(A, B, dA, dB, pu, ev, ep, &inside)) return -1;
        A = B;
        dA = dB;
    }
    return inside;
}

// The point's local (u, v) from the U/V model, with its error bound.
// Returns false when the point is outside the model window.
AGJ_HD bool model_uv_local(const FastModel& M, double lat, double lng, const PolyLocal& P, float* pu, float* pv,
                           float* dp) {
    float ah, al, bh, bl;
    if (!M.uv_enabled || !model_offsets(M, double_bits(lat), double_bits(lng), &ah, &al, &bh, &bl)) return false;
    float uth, utl, vth, vtl;
    model_eval_xy(M.uvl, M.uvh, M.f0uv, ah, al, bh, bl, &uth, &utl, &vth, &vtl);
    const float xu = ((float)(M.n0u - P.ru) + uth) + utl;
    const float xv = ((float)(M.n0v - P.rv) + vth) + vtl;
    *pu = xu;
    *pv = xv;
    *dp = M.err_uv + (fabs_f(xu) + fabs_f(xv)) * 2.4e-7f + 1e-5f;
    return true;
}

}  // namespace agj
