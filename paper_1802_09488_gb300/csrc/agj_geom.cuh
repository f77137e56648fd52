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

}  // namespace agj
