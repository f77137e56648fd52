/*
 * oracle.c — plain, slow, obviously-correct CPU oracle for the probe side of
 * the adaptive geospatial join (Kipf et al., "Adaptive Geospatial Joins for
 * Modern Hardware").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes (FP64, round-to-nearest, built with -ffp-contract=off so
 * that no multiply-add is fused; the only operations on the cell-id and PIP
 * paths are + - * / sqrt floor round and comparisons):
 *
 *   - sincos of an angle in degrees (own degree reduction + Taylor series;
 *     the paper is silent on the projection, §II "Google S2");
 *   - the point -> unit cube face -> (u,v) -> (s,t) -> (i,j) -> Hilbert
 *     position -> 64-bit cell id map (§II "Google S2": 3 face bits, up to 30
 *     bit pairs, one marker bit, zero tail);
 *   - ST_Covers of a point by a simple polygon (§II: points on edges or
 *     vertices are inside; "PIP": ray-crossing, odd count = inside), with
 *     geodesic edges, i.e. straight lines in the polygon's face (u,v) plane;
 *     polygons may have holes (rings after the outer one: the point is on
 *     the boundary if on any ring's edge, else inside if inside an odd
 *     number of rings), and ST_Contains (boundary excluded) is the interior
 *     of the same relation;
 *   - the exact join {(p, P) : P covers p} by brute force (bbox + uniform
 *     grid prefilter, then the full predicate) — §III-A: the exact join is
 *     the filter-and-refine result, which does not depend on the index;
 *   - the approximate join read off a logical covering ("super covering",
 *     §III-B) by the sorted-vector binary search of §II ("S2 stores the cell
 *     ids of a covering in a sorted vector ... binary search");
 *   - geodesic point-polygon distance and cell diagonals (§III-A: precision
 *     = max distance of a false-positive pair, bounded by the diagonal of the
 *     largest covering cell);
 *   - covering invariant checks (§II "interior cells are completely
 *     contained", §III-B "no overlap between the indexed cells").
 *
 * Parity status: every function here is pinned by tests under
 * tests/test_oracle_*.py (mpmath, closed forms, exhaustive small levels,
 * brute force, independent 3-D spherical predicates).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define OR_LEVELS 30
#define OR_EARTH_R 6371008.8
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* sincos in degrees                                                   */
/* ------------------------------------------------------------------ */

/* 1/k! for k = 0..18, each a single correctly rounded division of two
 * exactly representable doubles (18! < 2^53). */
static double g_inv_fact[19];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

static void or_init_consts(void) {
    double f = 1.0;
    g_inv_fact[0] = 1.0;
    for (int k = 1; k <= 18; ++k) {
        f = f * (double)k;          /* exact: k! < 2^53 */
        g_inv_fact[k] = 1.0 / f;
    }
}

/* pi/180 rounded to nearest double. */
static const double OR_DEG2RAD = 0x1.1df46a2529d39p-6;

/*
 * sin and cos of d degrees.
 *   q = round(d * fl(1/90))      (ties away from zero)
 *   r = d - 90 q                 (exact for |d| <= 225)
 *   x = r * fl(pi/180), z = x*x
 *   sin x: x + (x z) * h1, h8 = 1/17!, h_m = h_{m+1} z + (-1)^m / (2m+1)!
 *   cos x: 1 + z * g1,     g9 = -1/18!, g_m = g_{m+1} z + (-1)^m / (2m)!
 *   quadrant from q mod 4.
 */
void or_sincosd(double d, double *s_out, double *c_out) {
    pthread_once(&g_once, or_init_consts);
    double q = round(d * (1.0 / 90.0));
    double r = d - 90.0 * q;
    double x = r * OR_DEG2RAD;
    double z = x * x;

    double h = g_inv_fact[17];
    for (int m = 7; m >= 1; --m) {
        double c = g_inv_fact[2 * m + 1];
        if (m & 1) c = -c;
        h = h * z + c;
    }
    double sx = x + (x * z) * h;

    double g = -g_inv_fact[18];
    for (int m = 8; m >= 1; --m) {
        double c = g_inv_fact[2 * m];
        if (m & 1) c = -c;
        g = g * z + c;
    }
    double cx = 1.0 + z * g;

    long long qi = (long long)q;
    int n = (int)(((qi % 4) + 4) % 4);
    switch (n) {
    case 0: *s_out = sx;  *c_out = cx;  break;
    case 1: *s_out = cx;  *c_out = -sx; break;
    case 2: *s_out = -sx; *c_out = -cx; break;
    default: *s_out = -cx; *c_out = sx; break;
    }
}

/* ------------------------------------------------------------------ */
/* point -> face, (u,v)                                                */
/* ------------------------------------------------------------------ */

/* A point is valid iff lat and lng are finite, |lat| <= 90, |lng| <= 180. */
int or_point_valid(double lat, double lng) {
    if (!(lat == lat) || !(lng == lng)) return 0;
    if (!(fabs(lat) <= 90.0) || !(fabs(lng) <= 180.0)) return 0;
    return 1;
}

void or_latlng_xyz(double lat, double lng, double xyz[3]) {
    double sp, cp, sl, cl;
    or_sincosd(lat, &sp, &cp);
    or_sincosd(lng, &sl, &cl);
    xyz[0] = cp * cl;
    xyz[1] = cp * sl;
    xyz[2] = sp;
}

/* Face = axis of largest |component| (ties to the lower axis), +3 when
 * that component is negative.  (u,v) = ratio of the two other components
 * to the face component with S2's per-face axis order and signs. */
int or_xyz_face_uv(const double xyz[3], double *u, double *v) {
    double ax = fabs(xyz[0]), ay = fabs(xyz[1]), az = fabs(xyz[2]);
    int axis;
    if (ax >= ay && ax >= az) axis = 0;
    else if (ay >= az) axis = 1;
    else axis = 2;
    int face = axis + (xyz[axis] < 0.0 ? 3 : 0);
    double x = xyz[0], y = xyz[1], z = xyz[2];
    switch (face) {
    case 0: *u = y / x;    *v = z / x;    break;
    case 1: *u = -x / y;   *v = z / y;    break;
    case 2: *u = -x / z;   *v = -y / z;   break;
    case 3: *u = z / x;    *v = y / x;    break;
    case 4: *u = z / y;    *v = -x / y;   break;
    default: *u = -y / z;  *v = -x / z;   break;
    }
    return face;
}

/* Returns the face (0..5) or -1 for an invalid point. */
int or_face_uv(double lat, double lng, double *u, double *v) {
    if (!or_point_valid(lat, lng)) return -1;
    double xyz[3];
    or_latlng_xyz(lat, lng, xyz);
    return or_xyz_face_uv(xyz, u, v);
}

/* Quadratic (u -> s) projection and its inverse. */
double or_uv_to_st(double u) {
    if (u >= 0.0) return 0.5 * sqrt(1.0 + 3.0 * u);
    return 1.0 - 0.5 * sqrt(1.0 - 3.0 * u);
}

double or_st_to_uv(double s) {
    if (s >= 0.5) return ((4.0 * s) * s - 1.0) / 3.0;
    double w = 1.0 - s;
    return (1.0 - (4.0 * w) * w) / 3.0;
}

static uint32_t or_st_to_ij(double s) {
    double k = floor(s * 1073741824.0);   /* 2^30, exact scaling */
    if (k < 0.0) return 0u;
    if (k > 1073741823.0) return 1073741823u;
    return (uint32_t)k;
}

/* ------------------------------------------------------------------ */
/* Hilbert position and cell ids                                        */
/* ------------------------------------------------------------------ */
/*
 * Orientation o: bit 0 = swap i/j, bit 1 = invert both.  Start o = face & 1.
 * Per level, quadrant bits (ib, jb) are transformed by o (swap, then invert)
 * into the canonical frame where digits 0,1,2,3 visit (0,0),(0,1),(1,1),(1,0);
 * then o ^= 1 after digit 0, o ^= 3 after digit 3.
 */
uint64_t or_id_from_face_ij(int face, uint32_t i, uint32_t j) {
    uint64_t pos = 0;
    int o = face & 1;
    for (int lev = 1; lev <= OR_LEVELS; ++lev) {
        int sh = OR_LEVELS - lev;
        int ib = (int)((i >> sh) & 1u);
        int jb = (int)((j >> sh) & 1u);
        if (o & 1) { int t = ib; ib = jb; jb = t; }
        if (o & 2) { ib ^= 1; jb ^= 1; }
        int digit;
        if (ib == 0 && jb == 0) digit = 0;
        else if (ib == 0 && jb == 1) digit = 1;
        else if (ib == 1 && jb == 1) digit = 2;
        else digit = 3;
        pos = (pos << 2) | (uint64_t)digit;
        if (digit == 0) o ^= 1;
        else if (digit == 3) o ^= 3;
    }
    return ((uint64_t)face << 61) | (pos << 1) | 1ull;
}

/* Level of a cell id: 30 - (trailing zeros)/2. */
int or_id_level(uint64_t id) {
    if (id == 0) return -1;
    int tz = 0;
    while (((id >> tz) & 1ull) == 0) ++tz;
    return OR_LEVELS - tz / 2;
}

uint64_t or_id_parent(uint64_t id, int level) {
    uint64_t lsb = 1ull << (2 * (OR_LEVELS - level));
    return (id & ~(2 * lsb - 1)) | lsb;
}

uint64_t or_id_range_min(uint64_t id) {
    uint64_t lsb = id & (~id + 1);
    return id - (lsb - 1);
}

uint64_t or_id_range_max(uint64_t id) {
    uint64_t lsb = id & (~id + 1);
    return id + (lsb - 1);
}

/* Decode a cell id into face, level and the cell's (i, j) at that level. */
int or_id_decode(uint64_t id, int *face, int *level, uint32_t *i_out, uint32_t *j_out) {
    int lev = or_id_level(id);
    if (lev < 0) return -1;
    int f = (int)(id >> 61);
    if (f > 5) return -1;
    int o = f & 1;
    uint32_t i = 0, j = 0;
    for (int l = 1; l <= lev; ++l) {
        int digit = (int)((id >> (61 - 2 * l)) & 3ull);
        int ib, jb;
        switch (digit) {
        case 0: ib = 0; jb = 0; break;
        case 1: ib = 0; jb = 1; break;
        case 2: ib = 1; jb = 1; break;
        default: ib = 1; jb = 0; break;
        }
        /* undo: invert, then swap */
        if (o & 2) { ib ^= 1; jb ^= 1; }
        if (o & 1) { int t = ib; ib = jb; jb = t; }
        i = (i << 1) | (uint32_t)ib;
        j = (j << 1) | (uint32_t)jb;
        if (digit == 0) o ^= 1;
        else if (digit == 3) o ^= 3;
    }
    *face = f; *level = lev; *i_out = i; *j_out = j;
    return 0;
}

/* Leaf (level-30) cell id of a point; 0 for an invalid point. */
uint64_t or_cell_id(double lat, double lng) {
    double u, v;
    int face = or_face_uv(lat, lng, &u, &v);
    if (face < 0) return 0;
    uint32_t i = or_st_to_ij(or_uv_to_st(u));
    uint32_t j = or_st_to_ij(or_uv_to_st(v));
    return or_id_from_face_ij(face, i, j);
}

void or_cell_ids(const double *latlng, int64_t n, uint64_t *out) {
    for (int64_t k = 0; k < n; ++k) out[k] = or_cell_id(latlng[2 * k], latlng[2 * k + 1]);
}

/* (u_lo, u_hi, v_lo, v_hi) of a cell. */
int or_cell_uv_rect(uint64_t id, double rect[4]) {
    int face, lev; uint32_t i, j;
    if (or_id_decode(id, &face, &lev, &i, &j) != 0) return -1;
    double scale = ldexp(1.0, -lev);
    rect[0] = or_st_to_uv((double)i * scale);
    rect[1] = or_st_to_uv((double)(i + 1) * scale);
    rect[2] = or_st_to_uv((double)j * scale);
    rect[3] = or_st_to_uv((double)(j + 1) * scale);
    return face;
}

/* ------------------------------------------------------------------ */
/* geodesy (for the precision checks only; uses libm freely)           */
/* ------------------------------------------------------------------ */

static void or_face_uv_to_xyz(int face, double u, double v, double p[3]) {
    switch (face) {
    case 0: p[0] = 1.0;  p[1] = u;    p[2] = v;    break;
    case 1: p[0] = -u;   p[1] = 1.0;  p[2] = v;    break;
    case 2: p[0] = -u;   p[1] = -v;   p[2] = 1.0;  break;
    case 3: p[0] = -1.0; p[1] = -v;   p[2] = -u;   break;
    case 4: p[0] = v;    p[1] = -1.0; p[2] = -u;   break;
    default: p[0] = v;   p[1] = u;    p[2] = -1.0; break;
    }
    double n = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    p[0] /= n; p[1] /= n; p[2] /= n;
}

static void or_cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double or_dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double or_norm(const double a[3]) { return sqrt(or_dot(a, a)); }

static double or_angle(const double a[3], const double b[3]) {
    double c[3];
    or_cross(a, b, c);
    return atan2(or_norm(c), or_dot(a, b));
}

/* Great-circle distance in metres between two unit-cube face points. */
double or_uv_dist_m(int face, double u0, double v0, double u1, double v1) {
    double a[3], b[3];
    or_face_uv_to_xyz(face, u0, v0, a);
    or_face_uv_to_xyz(face, u1, v1, b);
    return OR_EARTH_R * or_angle(a, b);
}

/* Cell diagonal: the larger of the two great-circle corner-to-corner
 * distances. */
double or_cell_diag_m(uint64_t id) {
    double r[4];
    int face = or_cell_uv_rect(id, r);
    if (face < 0) return -1.0;
    double d1 = or_uv_dist_m(face, r[0], r[2], r[1], r[3]);
    double d2 = or_uv_dist_m(face, r[0], r[3], r[1], r[2]);
    return d1 > d2 ? d1 : d2;
}

/* Angle from unit vector p to the minor great-circle arc a-b. */
static double or_angle_point_arc(const double p[3], const double a[3], const double b[3]) {
    double n[3];
    or_cross(a, b, n);
    double nn = or_norm(n);
    double da = or_angle(p, a), db = or_angle(p, b);
    double best = da < db ? da : db;
    if (nn == 0.0) return best;
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    double pn = or_dot(p, n);
    double c[3] = {p[0] - pn * n[0], p[1] - pn * n[1], p[2] - pn * n[2]};
    double cn = or_norm(c);
    if (cn == 0.0) return best;
    c[0] /= cn; c[1] /= cn; c[2] /= cn;
    double t1[3], t2[3];
    or_cross(a, c, t1);
    or_cross(c, b, t2);
    if (or_dot(t1, n) >= 0.0 && or_dot(t2, n) >= 0.0) {
        double perp = atan2(fabs(pn), cn);
        if (perp < best) best = perp;
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* ST_Covers in the polygon's face (u,v) plane                          */
/* ------------------------------------------------------------------ */
/*
 * Ring rule for a closed ring uv[0..n-1] (implicitly closed) and a point
 * (pu, pv):
 *   for each edge (a,b):
 *     o = (b.u - a.u)*(p.v - a.v) - (b.v - a.v)*(p.u - a.u)
 *     o == 0 and p inside the edge's closed bbox      -> covered (boundary)
 *     (a.v <= p.v < b.v and o > 0) or
 *     (b.v <= p.v < a.v and o < 0)                     -> toggle
 *   odd number of toggles -> covered.
 */
int or_ring_relate_uv(const double *uv, int64_t n, double pu, double pv);
int or_rings_relate_uv(const double *uv, const int64_t *ring_off, int64_t n_rings, double pu, double pv);
int or_ring_covers_uv(const double *uv, int64_t n, double pu, double pv) {
    return or_ring_relate_uv(uv, n, pu, pv) != 0;
}

/* Where the point lies relative to the ring: 0 exterior, 1 on the boundary
 * (the on-edge case of the ring rule above), 2 interior (odd crossings and
 * on no edge).  ST_Covers (and ST_Intersects, which for a point and a
 * polygon is the same predicate) holds for 1 and 2; ST_Contains, which
 * excludes the boundary, for 2 only (§II: the paper's predicate is
 * ST_Covers; other predicates "can be implemented with similar
 * techniques"). */
int or_ring_relate_uv(const double *uv, int64_t n, double pu, double pv) {
    int inside = 0;
    for (int64_t k = 0; k < n; ++k) {
        const double *a = uv + 2 * k;
        const double *b = uv + 2 * ((k + 1) % n);
        double o = (b[0] - a[0]) * (pv - a[1]) - (b[1] - a[1]) * (pu - a[0]);
        double umin = a[0] < b[0] ? a[0] : b[0], umax = a[0] < b[0] ? b[0] : a[0];
        double vmin = a[1] < b[1] ? a[1] : b[1], vmax = a[1] < b[1] ? b[1] : a[1];
        if (o == 0.0 && pu >= umin && pu <= umax && pv >= vmin && pv <= vmax) return 1;
        if ((a[1] <= pv && pv < b[1] && o > 0.0) || (b[1] <= pv && pv < a[1] && o < 0.0))
            inside = !inside;
    }
    return inside ? 2 : 0;
}

/* A polygon set: vertices in (lat, lng) degrees.  Polygon k has the rings
 * pr[k] .. pr[k+1]-1 (the outer boundary first, then its holes), ring r the
 * vertices rv[r] .. rv[r+1]-1, each ring implicitly closed; a polygon's
 * vertices are contiguous, off[k] .. off[k+1]-1.  Prepared into face uv
 * once. */
typedef struct {
    int64_t n_polys;
    int64_t *off;          /* n_polys + 1 */
    int64_t *pr;           /* n_polys + 1 */
    int64_t *rv;           /* rings + 1 */
    double *uv;            /* 2 * off[n_polys] */
    int *face;             /* -1 if the polygon is not on a single face */
    double *bbox;          /* 4 per polygon: umin umax vmin vmax */
    /* uniform grid prefilter, one per face */
    int grid_n;
    double g_lo[6][2], g_step[6][2];
    int g_used[6];
    int64_t *g_start[6];   /* grid_n*grid_n + 1 */
    int32_t *g_items[6];
    int contains;          /* 0: ST_Covers / ST_Intersects, 1: ST_Contains (boundary excluded) */
    /* polygons whose vertices lie on more than one face (face[k] == OR_CAP):
     * each has a centre c (unit vector) and a tangent basis e1, e2; its
     * vertices are projected gnomonically about c into cap_uv, its bbox
     * there is bbox[4k..]; cap_ids lists them ascending */
    double *xyz;           /* 3 per vertex */
    double *cap_frame;     /* 9 per polygon: c, e1, e2 */
    double *cap_uv;        /* 2 per vertex (cap polygons only) */
    int64_t *cap_ids;
    int64_t n_caps;
} or_polyset;

/* face[k] of a polygon spanning cube faces (its vertices within
 * OR_CAP_COS of their normalised mean) */
#define OR_CAP 6
#define OR_CAP_COS 0.96592582628906831   /* cos 15 degrees */

static int or_cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void or_polyset_free(or_polyset *ps) {
    if (!ps) return;
    free(ps->off); free(ps->pr); free(ps->rv); free(ps->uv); free(ps->face); free(ps->bbox);
    free(ps->xyz); free(ps->cap_frame); free(ps->cap_uv); free(ps->cap_ids);
    for (int f = 0; f < 6; ++f) { free(ps->g_start[f]); free(ps->g_items[f]); }
    free(ps);
}

/* A polygon whose vertices lie on more than one cube face: its geodesic
 * edges are straight lines in any gnomonic projection whose centre sees all
 * of it, so the ring rule runs in the projection about the normalised mean
 * c of its vertices (a plane of the oracle's own, independent of the cube
 * faces).  Supported when every vertex is within 15 degrees of c (then the
 * polygon and any point tested lie well inside c's hemisphere).  Fills the
 * frame, the projected vertices and the bbox; returns OR_CAP or -1. */
static void or_cap_project(const double *frame, const double p[3], double *u, double *v) {
    double w = frame[0] * p[0] + frame[1] * p[1] + frame[2] * p[2];
    *u = (frame[3] * p[0] + frame[4] * p[1] + frame[5] * p[2]) / w;
    *v = (frame[6] * p[0] + frame[7] * p[1] + frame[8] * p[2]) / w;
}

static int or_cap_prepare(or_polyset *ps, int64_t k) {
    int64_t s = ps->off[k], e = ps->off[k + 1];
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t t = s; t < e; ++t) {
        const double *p = ps->xyz + 3 * t;
        if (!(p[0] == p[0])) return -1;          /* an invalid vertex */
        c[0] += p[0]; c[1] += p[1]; c[2] += p[2];
    }
    double n = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    if (!(n > 0.0)) return -1;
    c[0] /= n; c[1] /= n; c[2] /= n;
    for (int64_t t = s; t < e; ++t) {
        const double *p = ps->xyz + 3 * t;
        if (!(p[0] * c[0] + p[1] * c[1] + p[2] * c[2] >= OR_CAP_COS)) return -1;
    }
    /* e1 perpendicular to c (built from the axis least aligned with c), e2 = c x e1 */
    double a[3] = {0.0, 0.0, 0.0};
    int m = fabs(c[0]) <= fabs(c[1]) ? (fabs(c[0]) <= fabs(c[2]) ? 0 : 2) : (fabs(c[1]) <= fabs(c[2]) ? 1 : 2);
    a[m] = 1.0;
    double e1[3], e2[3];
    double d = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
    for (int q = 0; q < 3; ++q) e1[q] = a[q] - d * c[q];
    double ne = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int q = 0; q < 3; ++q) e1[q] /= ne;
    e2[0] = c[1] * e1[2] - c[2] * e1[1];
    e2[1] = c[2] * e1[0] - c[0] * e1[2];
    e2[2] = c[0] * e1[1] - c[1] * e1[0];
    double *f = ps->cap_frame + 9 * k;
    for (int q = 0; q < 3; ++q) { f[q] = c[q]; f[3 + q] = e1[q]; f[6 + q] = e2[q]; }
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int64_t t = s; t < e; ++t) {
        double u, v;
        or_cap_project(f, ps->xyz + 3 * t, &u, &v);
        ps->cap_uv[2 * t] = u; ps->cap_uv[2 * t + 1] = v;
        if (u < umin) umin = u;
        if (u > umax) umax = u;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
    }
    ps->bbox[4 * k] = umin; ps->bbox[4 * k + 1] = umax;
    ps->bbox[4 * k + 2] = vmin; ps->bbox[4 * k + 3] = vmax;
    ps->cap_ids[ps->n_caps++] = k;
    return OR_CAP;
}

or_polyset *or_polyset_new_rings(const double *latlng, const int64_t *ring_off, const int64_t *poly_ring_off,
                                 int64_t n_polys, int grid_n) {
    or_polyset *ps = (or_polyset *)calloc(1, sizeof(or_polyset));
    ps->n_polys = n_polys;
    int64_t n_rings = poly_ring_off[n_polys];
    ps->pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_polys + 1));
    memcpy(ps->pr, poly_ring_off, sizeof(int64_t) * (size_t)(n_polys + 1));
    ps->rv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_rings + 1));
    memcpy(ps->rv, ring_off, sizeof(int64_t) * (size_t)(n_rings + 1));
    ps->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_polys + 1));
    for (int64_t k = 0; k <= n_polys; ++k) ps->off[k] = ring_off[poly_ring_off[k]];
    const int64_t *off = ps->off;
    {
        int64_t nvv = off[n_polys] > 0 ? off[n_polys] : 1;
        ps->xyz = (double *)malloc(sizeof(double) * 3 * (size_t)nvv);
        ps->cap_uv = (double *)calloc(2 * (size_t)nvv, sizeof(double));
        ps->cap_frame = (double *)calloc(9 * (size_t)(n_polys > 0 ? n_polys : 1), sizeof(double));
        ps->cap_ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_polys > 0 ? n_polys : 1));
        ps->n_caps = 0;
        for (int64_t t = 0; t < off[n_polys]; ++t)
            if (or_point_valid(latlng[2 * t], latlng[2 * t + 1])) or_latlng_xyz(latlng[2 * t], latlng[2 * t + 1], ps->xyz + 3 * t);
            else ps->xyz[3 * t] = ps->xyz[3 * t + 1] = ps->xyz[3 * t + 2] = NAN;
    }
    int64_t nv = off[n_polys];
    ps->uv = (double *)malloc(sizeof(double) * 2 * (size_t)(nv > 0 ? nv : 1));
    ps->face = (int *)malloc(sizeof(int) * (size_t)(n_polys > 0 ? n_polys : 1));
    ps->bbox = (double *)malloc(sizeof(double) * 4 * (size_t)(n_polys > 0 ? n_polys : 1));
    for (int64_t k = 0; k < n_polys; ++k) {
        int face = -2;
        double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        for (int64_t t = off[k]; t < off[k + 1]; ++t) {
            double u, v;
            int f = or_face_uv(latlng[2 * t], latlng[2 * t + 1], &u, &v);
            if (f < 0 || (face != -2 && f != face)) face = -1;
            else if (face == -2) face = f;
            ps->uv[2 * t] = u; ps->uv[2 * t + 1] = v;
            if (u < umin) umin = u;
            if (u > umax) umax = u;
            if (v < vmin) vmin = v;
            if (v > vmax) vmax = v;
        }
        int bad = ps->pr[k + 1] <= ps->pr[k];
        for (int64_t r = ps->pr[k]; r < ps->pr[k + 1]; ++r)
            if (ps->rv[r + 1] - ps->rv[r] < 3) bad = 1;
        ps->bbox[4 * k] = umin; ps->bbox[4 * k + 1] = umax;
        ps->bbox[4 * k + 2] = vmin; ps->bbox[4 * k + 3] = vmax;
        if (face == -1 && !bad) face = or_cap_prepare(ps, k);
        ps->face[k] = (face < 0 || bad) ? -1 : face;
    }
    /* uniform grid per face over the union of the polygons' bboxes; each
     * polygon is registered in every grid cell its bbox, widened by 1e-9,
     * overlaps, so that rounding in the grid-cell computation of a point
     * never drops a polygon whose closed bbox holds the point. */
    ps->grid_n = grid_n < 1 ? 1 : grid_n;
    int G = ps->grid_n;
    const double W = 1e-9;
    for (int f = 0; f < 6; ++f) {
        double lo0 = INFINITY, hi0 = -INFINITY, lo1 = INFINITY, hi1 = -INFINITY;
        for (int64_t k = 0; k < n_polys; ++k) {
            if (ps->face[k] != f) continue;
            const double *bb = ps->bbox + 4 * k;
            if (bb[0] < lo0) lo0 = bb[0];
            if (bb[1] > hi0) hi0 = bb[1];
            if (bb[2] < lo1) lo1 = bb[2];
            if (bb[3] > hi1) hi1 = bb[3];
        }
        if (!(lo0 <= hi0)) { ps->g_used[f] = 0; continue; }
        ps->g_used[f] = 1;
        lo0 -= 2 * W; hi0 += 2 * W; lo1 -= 2 * W; hi1 += 2 * W;
        ps->g_lo[f][0] = lo0; ps->g_lo[f][1] = lo1;
        ps->g_step[f][0] = (hi0 - lo0) / G;
        ps->g_step[f][1] = (hi1 - lo1) / G;
        int64_t *cnt = (int64_t *)calloc((size_t)G * G + 1, sizeof(int64_t));
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                int64_t acc = 0;
                for (int64_t c = 0; c < (int64_t)G * G; ++c) { int64_t t = cnt[c]; cnt[c] = acc; acc += t; }
                cnt[(int64_t)G * G] = acc;
                ps->g_start[f] = (int64_t *)malloc(sizeof(int64_t) * ((size_t)G * G + 1));
                memcpy(ps->g_start[f], cnt, sizeof(int64_t) * ((size_t)G * G + 1));
                ps->g_items[f] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(acc > 0 ? acc : 1));
            }
            for (int64_t k = 0; k < n_polys; ++k) {
                if (ps->face[k] != f) continue;
                const double *bb = ps->bbox + 4 * k;
                int a0 = (int)floor((bb[0] - W - lo0) / ps->g_step[f][0]);
                int a1 = (int)floor((bb[1] + W - lo0) / ps->g_step[f][0]);
                int b0 = (int)floor((bb[2] - W - lo1) / ps->g_step[f][1]);
                int b1 = (int)floor((bb[3] + W - lo1) / ps->g_step[f][1]);
                if (a0 < 0) a0 = 0;
                if (b0 < 0) b0 = 0;
                if (a1 > G - 1) a1 = G - 1;
                if (b1 > G - 1) b1 = G - 1;
                for (int a = a0; a <= a1; ++a)
                    for (int b = b0; b <= b1; ++b) {
                        int64_t c = (int64_t)a * G + b;
                        if (pass == 0) cnt[c]++;
                        else ps->g_items[f][cnt[c]++] = (int32_t)k;
                    }
            }
        }
        free(cnt);
        /* sort each cell's list so that hits come out in ascending order */
        for (int64_t c = 0; c < (int64_t)G * G; ++c) {
            int64_t s = ps->g_start[f][c], e = ps->g_start[f][c + 1];
            qsort(ps->g_items[f] + s, (size_t)(e - s), sizeof(int32_t), or_cmp_i32);
        }
    }
    return ps;
}

/* The same relation for rings given directly in uv: ring q spans the
 * vertices ring_off[q] .. ring_off[q+1]-1 of uv (n_rings rings). */
int or_rings_relate_uv(const double *uv, const int64_t *ring_off, int64_t n_rings, double pu, double pv) {
    int parity = 0;
    for (int64_t q = 0; q < n_rings; ++q) {
        int rel = or_ring_relate_uv(uv + 2 * ring_off[q], ring_off[q + 1] - ring_off[q], pu, pv);
        if (rel == 1) return 1;
        if (rel == 2) parity ^= 1;
    }
    return parity ? 2 : 0;
}

/* Every polygon a single ring: polygon k = latlng[2*off[k] .. 2*off[k+1]). */
or_polyset *or_polyset_new(const double *latlng, const int64_t *off, int64_t n_polys, int grid_n) {
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_polys + 1));
    for (int64_t k = 0; k <= n_polys; ++k) pr[k] = k;
    or_polyset *ps = or_polyset_new_rings(latlng, off, pr, n_polys, grid_n);
    free(pr);
    return ps;
}

int or_polyset_face(const or_polyset *ps, int64_t k) { return ps->face[k]; }

/* Relation of a point (in the polygon's face uv) to polygon k with all its
 * rings: on the boundary (1) if it lies on an edge of any ring, else interior
 * (2) if it is inside an odd number of rings (outer boundary minus holes),
 * else exterior (0). */
int or_polygon_relate_uv(const or_polyset *ps, int64_t k, double u, double v) {
    return or_rings_relate_uv(ps->uv, ps->rv + ps->pr[k], ps->pr[k + 1] - ps->pr[k], u, v);
}

/* Selects the join predicate of the set: 0 ST_Covers (ST_Intersects is the
 * same predicate for a point), 1 ST_Contains. */
void or_polyset_set_contains(or_polyset *ps, int contains) { ps->contains = contains ? 1 : 0; }

/* The set's predicate for a point already in face (u,v) on the polygon's
 * face. */
static int or_pred_uv(const or_polyset *ps, int64_t k, double u, double v) {
    const double *bb = ps->bbox + 4 * k;
    if (!(u >= bb[0] && u <= bb[1] && v >= bb[2] && v <= bb[3])) return 0;
    int rel = or_polygon_relate_uv(ps, k, u, v);
    return ps->contains ? rel == 2 : rel != 0;
}

/* The set's predicate for a polygon spanning faces (OR_CAP) and a point
 * given by its unit vector: in the polygon's own gnomonic plane. */
static int or_pred_cap(const or_polyset *ps, int64_t k, const double p[3]) {
    const double *f = ps->cap_frame + 9 * k;
    if (!(p[0] * f[0] + p[1] * f[1] + p[2] * f[2] > 0.5)) return 0;   /* > 60 degrees from the centre: outside */
    double u, v;
    or_cap_project(f, p, &u, &v);
    const double *bb = ps->bbox + 4 * k;
    if (!(u >= bb[0] && u <= bb[1] && v >= bb[2] && v <= bb[3])) return 0;
    int rel = or_rings_relate_uv(ps->cap_uv, ps->rv + ps->pr[k], ps->pr[k + 1] - ps->pr[k], u, v);
    return ps->contains ? rel == 2 : rel != 0;
}

/* ST_Covers(P_k, p) (or ST_Contains with the set's predicate): same face,
 * inside the closed uv bbox, ring rule; a polygon spanning faces in its own
 * gnomonic plane. */
int or_polygon_covers(const or_polyset *ps, int64_t k, double lat, double lng) {
    if (ps->face[k] == OR_CAP) {
        if (!or_point_valid(lat, lng)) return 0;
        double p[3];
        or_latlng_xyz(lat, lng, p);
        return or_pred_cap(ps, k, p);
    }
    double u, v;
    int f = or_face_uv(lat, lng, &u, &v);
    if (f < 0 || f != ps->face[k]) return 0;
    return or_pred_uv(ps, k, u, v);
}

/* Candidate polygons for a point via the grid (ascending ids).  Returns the
 * count and a pointer into the grid lists. */
static int64_t or_grid_candidates(const or_polyset *ps, int f, double u, double v, const int32_t **items) {
    if (f < 0 || !ps->g_used[f]) return 0;
    int G = ps->grid_n;
    double a = floor((u - ps->g_lo[f][0]) / ps->g_step[f][0]);
    double b = floor((v - ps->g_lo[f][1]) / ps->g_step[f][1]);
    if (!(a >= 0.0 && a < G && b >= 0.0 && b < G)) return 0;
    int64_t c = (int64_t)a * G + (int64_t)b;
    *items = ps->g_items[f] + ps->g_start[f][c];
    return ps->g_start[f][c + 1] - ps->g_start[f][c];
}

static int64_t or_point_hits(const or_polyset *ps, double lat, double lng, uint32_t *out) {
    double u, v;
    int f = or_face_uv(lat, lng, &u, &v);
    if (f < 0) return 0;
    const int32_t *items = NULL;
    int64_t m = or_grid_candidates(ps, f, u, v, &items);
    int64_t cnt = 0;
    for (int64_t t = 0; t < m; ++t) {
        int32_t k = items[t];
        if (or_pred_uv(ps, k, u, v)) {
            if (out) out[cnt] = (uint32_t)k;
            ++cnt;
        }
    }
    if (ps->n_caps) {
        /* polygons spanning faces: every one, then merged in ascending order */
        double p[3];
        or_latlng_xyz(lat, lng, p);
        for (int64_t t = 0; t < ps->n_caps; ++t) {
            int64_t k = ps->cap_ids[t];
            if (!or_pred_cap(ps, k, p)) continue;
            if (out) {
                int64_t b = cnt - 1;
                while (b >= 0 && out[b] > (uint32_t)k) { out[b + 1] = out[b]; --b; }
                out[b + 1] = (uint32_t)k;
            }
            ++cnt;
        }
    }
    return cnt;
}

/* Brute force over every polygon, no grid: the definition itself. */
int64_t or_point_hits_brute(const or_polyset *ps, double lat, double lng, uint32_t *out) {
    int64_t cnt = 0;
    for (int64_t k = 0; k < ps->n_polys; ++k) {
        if (or_polygon_covers(ps, k, lat, lng)) {
            if (out) out[cnt] = (uint32_t)k;
            ++cnt;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* threaded joins producing CSR (offsets u64[n+1], ids u32[nnz])        */
/* ------------------------------------------------------------------ */

typedef struct {
    int mode;                 /* 0 exact (brute force), 1 approx (logical covering) */
    const or_polyset *ps;
    const double *pts;
    int64_t lo, hi;
    uint64_t *counts;         /* pass 0 */
    const uint64_t *offsets;  /* pass 1 */
    uint32_t *ids;
    int pass;
    /* logical covering */
    const uint64_t *cells; int64_t n_cells;
    const uint64_t *ref_off; const uint32_t *refs;
} or_job;

/* Sorted-vector probe: index of the unique cell whose range holds `id`,
 * or -1. */
int64_t or_logical_find(const uint64_t *cells, int64_t m, uint64_t id) {
    int64_t lo = 0, hi = m;   /* first cell with range_min > id */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (or_id_range_min(cells[mid]) <= id) lo = mid + 1;
        else hi = mid;
    }
    int64_t k = lo - 1;
    if (k < 0) return -1;
    if (id <= or_id_range_max(cells[k])) return k;
    return -1;
}

static int64_t or_point_approx(const or_job *jb, double lat, double lng, uint32_t *out) {
    uint64_t id = or_cell_id(lat, lng);
    if (id == 0) return 0;
    int64_t k = or_logical_find(jb->cells, jb->n_cells, id);
    if (k < 0) return 0;
    int64_t cnt = 0;
    for (uint64_t t = jb->ref_off[k]; t < jb->ref_off[k + 1]; ++t) {
        if (out) out[cnt] = jb->refs[t] >> 1;
        ++cnt;
    }
    if (out) {   /* ascending polygon ids (insertion sort, short lists) */
        for (int64_t a = 1; a < cnt; ++a) {
            uint32_t x = out[a]; int64_t b = a - 1;
            while (b >= 0 && out[b] > x) { out[b + 1] = out[b]; --b; }
            out[b + 1] = x;
        }
    }
    return cnt;
}

static void *or_job_run(void *arg) {
    or_job *jb = (or_job *)arg;
    for (int64_t p = jb->lo; p < jb->hi; ++p) {
        double lat = jb->pts[2 * p], lng = jb->pts[2 * p + 1];
        uint32_t *dst = jb->pass ? jb->ids + jb->offsets[p] : NULL;
        int64_t c = jb->mode == 0 ? or_point_hits(jb->ps, lat, lng, dst)
                                  : or_point_approx(jb, lat, lng, dst);
        if (!jb->pass) jb->counts[p] = (uint64_t)c;
    }
    return NULL;
}

static int or_nthreads(int req) {
    if (req > 0) return req;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Runs one pass over [0, n) split across threads. */
static void or_run_pass(or_job proto, int64_t n, int nt) {
    if (nt > 256) nt = 256;
    pthread_t th[256];
    or_job jobs[256];
    int64_t chunk = (n + nt - 1) / nt;
    int used = 0;
    for (int t = 0; t < nt; ++t) {
        int64_t lo = (int64_t)t * chunk, hi = lo + chunk;
        if (lo >= n) break;
        if (hi > n) hi = n;
        jobs[t] = proto; jobs[t].lo = lo; jobs[t].hi = hi;
        pthread_create(&th[t], NULL, or_job_run, &jobs[t]);
        ++used;
    }
    for (int t = 0; t < used; ++t) pthread_join(th[t], NULL);
}

/* Counting pass: offsets[0..n] (exclusive scan of per-point counts);
 * returns nnz.  Then call or_join_fill with an ids buffer of nnz. */
static uint64_t or_join_count(or_job proto, int64_t n, uint64_t *offsets, int nt) {
    proto.pass = 0;
    proto.counts = offsets;   /* counts land in offsets[0..n-1] first */
    or_run_pass(proto, n, nt);
    uint64_t acc = 0;
    for (int64_t p = 0; p < n; ++p) { uint64_t c = offsets[p]; offsets[p] = acc; acc += c; }
    offsets[n] = acc;
    return acc;
}

static void or_join_fill(or_job proto, int64_t n, const uint64_t *offsets, uint32_t *ids, int nt) {
    proto.pass = 1;
    proto.offsets = offsets;
    proto.ids = ids;
    or_run_pass(proto, n, nt);
}

uint64_t or_join_exact_count(const or_polyset *ps, const double *pts, int64_t n, uint64_t *offsets, int nt) {
    or_job j; memset(&j, 0, sizeof j);
    j.mode = 0; j.ps = ps; j.pts = pts;
    return or_join_count(j, n, offsets, or_nthreads(nt));
}

void or_join_exact_fill(const or_polyset *ps, const double *pts, int64_t n, const uint64_t *offsets, uint32_t *ids, int nt) {
    or_job j; memset(&j, 0, sizeof j);
    j.mode = 0; j.ps = ps; j.pts = pts;
    or_join_fill(j, n, offsets, ids, or_nthreads(nt));
}

uint64_t or_join_approx_count(const uint64_t *cells, int64_t m, const uint64_t *ref_off, const uint32_t *refs,
                              const double *pts, int64_t n, uint64_t *offsets, int nt) {
    or_job j; memset(&j, 0, sizeof j);
    j.mode = 1; j.pts = pts; j.cells = cells; j.n_cells = m; j.ref_off = ref_off; j.refs = refs;
    return or_join_count(j, n, offsets, or_nthreads(nt));
}

void or_join_approx_fill(const uint64_t *cells, int64_t m, const uint64_t *ref_off, const uint32_t *refs,
                         const double *pts, int64_t n, const uint64_t *offsets, uint32_t *ids, int nt) {
    or_job j; memset(&j, 0, sizeof j);
    j.mode = 1; j.pts = pts; j.cells = cells; j.n_cells = m; j.ref_off = ref_off; j.refs = refs;
    or_join_fill(j, n, offsets, ids, or_nthreads(nt));
}

/* ------------------------------------------------------------------ */
/* geodesic distance point -> polygon                                   */
/* ------------------------------------------------------------------ */

/* 0 if the polygon covers the point, else the great-circle distance in
 * metres to its boundary (geodesic edges).  -1 for an invalid input. */
double or_dist_point_polygon_m(const or_polyset *ps, int64_t k, double lat, double lng) {
    if (!or_point_valid(lat, lng) || ps->face[k] < 0) return -1.0;
    if (or_polygon_covers(ps, k, lat, lng)) return 0.0;
    double p[3];
    {
        /* libm is fine here: this is a metric check, not a bit-exact path */
        double la = lat * (OR_PI / 180.0), lo = lng * (OR_PI / 180.0);
        p[0] = cos(la) * cos(lo); p[1] = cos(la) * sin(lo); p[2] = sin(la);
    }
    int f = ps->face[k];
    double best = INFINITY;
    for (int64_t r = ps->pr[k]; r < ps->pr[k + 1]; ++r) {
        int64_t s = ps->rv[r], nv = ps->rv[r + 1] - s;
        for (int64_t t = 0; t < nv; ++t) {
            double A[3], B[3];
            if (f == OR_CAP) {
                const double *a = ps->xyz + 3 * (s + t), *b = ps->xyz + 3 * (s + (t + 1) % nv);
                for (int q = 0; q < 3; ++q) { A[q] = a[q]; B[q] = b[q]; }
            } else {
                const double *a = ps->uv + 2 * (s + t);
                const double *b = ps->uv + 2 * (s + (t + 1) % nv);
                or_face_uv_to_xyz(f, a[0], a[1], A);
                or_face_uv_to_xyz(f, b[0], b[1], B);
            }
            double ang = or_angle_point_arc(p, A, B);
            if (ang < best) best = ang;
        }
    }
    return best * OR_EARTH_R;
}

/* ------------------------------------------------------------------ */
/* covering invariants                                                  */
/* ------------------------------------------------------------------ */

/* Does the closed segment a-b meet the closed axis-aligned rectangle r? */
static int or_seg_meets_rect(const double a[2], const double b[2], const double r[4]) {
    /* Liang-Barsky clipping of the parametric segment against the rect */
    double t0 = 0.0, t1 = 1.0;
    double d[2] = {b[0] - a[0], b[1] - a[1]};
    double lo[2] = {r[0], r[2]}, hi[2] = {r[1], r[3]};
    for (int ax = 0; ax < 2; ++ax) {
        if (d[ax] == 0.0) {
            if (a[ax] < lo[ax] || a[ax] > hi[ax]) return 0;
        } else {
            double ta = (lo[ax] - a[ax]) / d[ax];
            double tb = (hi[ax] - a[ax]) / d[ax];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
            if (t0 > t1) return 0;
        }
    }
    return 1;
}

/* Does an edge of any ring meet the closed rectangle r?  Ring q spans the
 * vertices ring_off[q] .. ring_off[q+1]-1 of uv. */
static int or_rings_meet_rect(const double *uv0, const int64_t *ring_off, int64_t n_rings, const double r[4]) {
    for (int64_t q = 0; q < n_rings; ++q) {
        const double *uv = uv0 + 2 * ring_off[q];
        int64_t nv = ring_off[q + 1] - ring_off[q];
        for (int64_t e = 0; e < nv; ++e)
            if (or_seg_meets_rect(uv + 2 * e, uv + 2 * ((e + 1) % nv), r)) return 1;
    }
    return 0;
}

/* The (u,v) of a point given by its unit vector on the plane of `face`
 * (the face's gnomonic coordinates, also beyond the face's square); 0 when
 * the point is not in the face's open hemisphere. */
static int or_xyz_uv_on_face(int face, const double xyz[3], double *u, double *v) {
    double x = xyz[0], y = xyz[1], z = xyz[2];
    switch (face) {
    case 0: if (!(x > 0.0)) return 0; *u = y / x;  *v = z / x;  break;
    case 1: if (!(y > 0.0)) return 0; *u = -x / y; *v = z / y;  break;
    case 2: if (!(z > 0.0)) return 0; *u = -x / z; *v = -y / z; break;
    case 3: if (!(x < 0.0)) return 0; *u = z / x;  *v = y / x;  break;
    case 4: if (!(y < 0.0)) return 0; *u = z / y;  *v = -x / y; break;
    default: if (!(z < 0.0)) return 0; *u = -y / z; *v = -x / z; break;
    }
    return 1;
}

/* report[0] = overlapping neighbour pairs (disjointness),
 * report[1] = true refs whose cell is not wholly inside the polygon,
 * report[2] = candidate refs whose cell, widened by cand_margin in (u,v),
 *             misses the polygon,
 * report[3] = candidate cells with diagonal >= eps (if eps_m > 0),
 * report[4] = refs to unknown polygons or cells off the polygon's face. */
void or_check_covering(const or_polyset *ps, const uint64_t *cells, int64_t m, const uint64_t *ref_off,
                       const uint32_t *refs, double eps_m, double cand_margin, int64_t report[5]) {
    for (int t = 0; t < 5; ++t) report[t] = 0;
    for (int64_t c = 0; c + 1 < m; ++c)
        if (or_id_range_max(cells[c]) >= or_id_range_min(cells[c + 1])) report[0]++;
    for (int64_t c = 0; c < m; ++c) {
        double r[4];
        int face = or_cell_uv_rect(cells[c], r);
        int has_cand = 0;
        for (uint64_t t = ref_off[c]; t < ref_off[c + 1]; ++t) {
            uint32_t pid = refs[t] >> 1;
            int interior = (int)(refs[t] & 1u);
            if ((int64_t)pid >= ps->n_polys || (ps->face[pid] != face && ps->face[pid] != OR_CAP)) {
                report[4]++;
                continue;
            }
            /* the polygon's rings in the cell's face coordinates: stored for a
             * one-face polygon, projected onto the face for one spanning faces */
            int64_t v0 = ps->off[pid], nv = ps->off[pid + 1] - v0;
            int64_t nr = ps->pr[pid + 1] - ps->pr[pid];
            const double *uv = ps->uv + 2 * v0;
            double *tmp = NULL;
            int64_t *roff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nr + 1));
            for (int64_t q = 0; q <= nr; ++q) roff[q] = ps->rv[ps->pr[pid] + q] - v0;
            if (ps->face[pid] == OR_CAP) {
                tmp = (double *)malloc(sizeof(double) * 2 * (size_t)nv);
                int ok = 1;
                for (int64_t t = 0; t < nv && ok; ++t)
                    ok = or_xyz_uv_on_face(face, ps->xyz + 3 * (v0 + t), tmp + 2 * t, tmp + 2 * t + 1);
                if (!ok) { report[4]++; free(tmp); free(roff); continue; }
                uv = tmp;
            }
            double cu = 0.5 * (r[0] + r[1]), cv = 0.5 * (r[2] + r[3]);
            int center_in = or_rings_relate_uv(uv, roff, nr, cu, cv) != 0;
            if (interior) {
                int meets = or_rings_meet_rect(uv, roff, nr, r);
                if (meets || !center_in) report[1]++;
            } else {
                has_cand = 1;
                double w[4] = {r[0] - cand_margin, r[1] + cand_margin, r[2] - cand_margin, r[3] + cand_margin};
                int meets = or_rings_meet_rect(uv, roff, nr, w), vertex_in = 0;
                for (int64_t e = 0; e < nv && !vertex_in; ++e)
                    vertex_in = uv[2 * e] >= w[0] && uv[2 * e] <= w[1] && uv[2 * e + 1] >= w[2] && uv[2 * e + 1] <= w[3];
                if (!meets && !center_in && !vertex_in) report[2]++;
            }
            free(tmp);
            free(roff);
        }
        if (eps_m > 0.0 && has_cand && !(or_cell_diag_m(cells[c]) < eps_m)) report[3]++;
    }
}
