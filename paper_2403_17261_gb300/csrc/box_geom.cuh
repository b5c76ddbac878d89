// box_geom.cuh -- contact geometry of boxes (FP64), for the box and plank
// bodies of the paper's Building and Bridge scenes (Section 6): box-plane,
// sphere-box and box-box (separating axes of two oriented boxes, then a
// clipped face manifold of up to 4 points or one edge point).  The
// functions are __host__ __device__ and use only IEEE-rounded operations
// (no rsqrt, no implicit contraction in the files that include this), so
// host and device runs give the same bits.
//
// Conventions: the normal points from the first shape towards the second;
// gap > 0 when apart; a contact when gap <= margin; quaternions as float4
// (x = w, y..w = vector part).  Decisions with a tolerance, so that exactly
// aligned boxes (which tie in exact arithmetic) decide the same in any
// precision accurate to well under it:
//  - axes: scanning A's faces, B's faces, then a_i x b_j (i major), a later
//    axis replaces the best so far only if its separation is larger by more
//    than kTieLen (0.3 mm); an a_i x b_j axis exists when |a_i x b_j| >
//    kEdgeMin; an edge axis is taken over the best face axis only if its
//    separation exceeds the face's by more than 5 % of the face's magnitude
//    + 0.01 x the smallest half extent;
//  - the incident face: the most anti-parallel, a later face winning only by
//    more than kTieDir in |cosine|;
//  - a sphere's centre inside a box: the least-penetrated face, a later face
//    winning only by more than kTieLen;
//  - clipping keeps points within kTieLen outside a reference side plane;
//  - the 4 deepest: k times, among the remaining candidates in order, the
//    first whose gap is within kTieLen of the smallest remaining gap.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace ovl {
namespace box {

#define OVL_HD __host__ __device__ __forceinline__

// ---- FP32 helpers (rows) ---------------------------------------------------
OVL_HD float3 v3(float x, float y, float z) { return make_float3(x, y, z); }
OVL_HD float3 add(float3 a, float3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
OVL_HD float3 sub(float3 a, float3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
OVL_HD float3 scl(float3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
OVL_HD float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
OVL_HD float3 crs(float3 a, float3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
OVL_HD float comp(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---- FP64 helpers (contact geometry) ---------------------------------------
OVL_HD double3 d3(double x, double y, double z) { return make_double3(x, y, z); }
OVL_HD double3 add(double3 a, double3 b) { return d3(a.x + b.x, a.y + b.y, a.z + b.z); }
OVL_HD double3 sub(double3 a, double3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
OVL_HD double3 scl(double3 a, double s) { return d3(a.x * s, a.y * s, a.z * s); }
OVL_HD double dot(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
OVL_HD double3 crs(double3 a, double3 b) { return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
OVL_HD double comp(double3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
OVL_HD float3 to_f(double3 a) { return make_float3((float)a.x, (float)a.y, (float)a.z); }
OVL_HD double3 to_d(float3 a) { return d3(a.x, a.y, a.z); }

constexpr double kTieLen = 3e-4;
constexpr double kTieDir = 1e-4;
constexpr double kEdgeMin = 1e-3;

// an oriented box: centre, world directions of its three axes, half extents
struct Obb {
    double3 c, u[3];
    double h[3];
};

// from an FP32 pose (centre, unit quaternion as float4 (w, x, y, z)) and
// half extents, widened exactly
OVL_HD Obb make_obb(float3 cf, float4 qf, float3 hf) {
    const double w = qf.x, x = qf.y, y = qf.z, z = qf.w;
    Obb b;
    b.c = to_d(cf);
    b.u[0] = d3(1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y + w * z), 2.0 * (x * z - w * y));
    b.u[1] = d3(2.0 * (x * y - w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z + w * x));
    b.u[2] = d3(2.0 * (x * z + w * y), 2.0 * (y * z - w * x), 1.0 - 2.0 * (x * x + y * y));
    b.h[0] = hf.x; b.h[1] = hf.y; b.h[2] = hf.z;
    return b;
}

// point of the box for local coordinates (a, b, c)
OVL_HD double3 at(const Obb &B, double a, double b, double c) {
    return add(B.c, add(add(scl(B.u[0], a), scl(B.u[1], b)), scl(B.u[2], c)));
}

// candidates (points, gaps) kept: k times, the first remaining candidate
// (in order) whose gap is within kTieLen of the smallest remaining gap;
// n <= 16, written back compacted in the order taken
OVL_HD int keep_deepest(double3 *P, double *G, int n, int k) {
    for (int i = 0; i < n && i < k; ++i) {
        double gmin = G[i];
        for (int j = i + 1; j < n; ++j) gmin = G[j] < gmin ? G[j] : gmin;
        int m = i;
        while (m < n - 1 && !(G[m] <= gmin + kTieLen)) ++m;   // bounded even with NaN gaps
        if (m != i) {
            // rotate [i, m] right by one so that the others keep their order
            const double3 pm = P[m];
            const double gm = G[m];
            for (int j = m; j > i; --j) { P[j] = P[j - 1]; G[j] = G[j - 1]; }
            P[i] = pm;
            G[i] = gm;
        }
    }
    return n < k ? n : k;
}

// Box (first) against the plane n.x = d (plane = (n, d), n unit, out of the
// solid).  normal = -n.  Returns the count (<= 4).
OVL_HD int box_plane(const Obb &B, float4 plane, double margin, double3 pts[4], double gaps[4], double3 &normal) {
    const double3 n = d3(plane.x, plane.y, plane.z);
    double3 P[8];
    double G[8];
    int m = 0;
    for (int v = 0; v < 8; ++v) {
        const double3 p = at(B, (v & 1) ? B.h[0] : -B.h[0], (v & 2) ? B.h[1] : -B.h[1], (v & 4) ? B.h[2] : -B.h[2]);
        const double g = dot(n, p) - (double)plane.w;
        if (g <= margin) { P[m] = p; G[m] = g; ++m; }
    }
    m = keep_deepest(P, G, m, 4);
    for (int i = 0; i < m; ++i) { pts[i] = P[i]; gaps[i] = G[i]; }
    normal = scl(n, -1.0);
    return m;
}

// Sphere (first: centre s, radius r) against a box (second): the point of
// the box nearest the centre, or with the centre inside its projection on
// the face of least penetration (a later face winning only by more than
// kTieLen).  Returns 1 when gap <= margin (outputs are written either way).
OVL_HD int sphere_box(double3 s, double r, const Obb &B, double margin, double3 &pt, double3 &normal, double &gap) {
    const double3 d = sub(s, B.c);
    double loc[3], cl[3];
    bool inside = true;
    for (int k = 0; k < 3; ++k) {
        loc[k] = dot(d, B.u[k]);
        cl[k] = loc[k] < -B.h[k] ? -B.h[k] : (loc[k] > B.h[k] ? B.h[k] : loc[k]);
        if (cl[k] != loc[k]) inside = false;
    }
    double3 nb;                                       // box -> sphere, world
    if (!inside) {
        const double e0 = loc[0] - cl[0], e1 = loc[1] - cl[1], e2 = loc[2] - cl[2];
        const double len = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        nb = add(add(scl(B.u[0], e0 / len), scl(B.u[1], e1 / len)), scl(B.u[2], e2 / len));
        gap = len - r;
    } else {
        int k = 0;
        double pen = B.h[0] - fabs(loc[0]);
        for (int j = 1; j < 3; ++j) {
            const double pj = B.h[j] - fabs(loc[j]);
            if (pj < pen - kTieLen) { pen = pj; k = j; }
        }
        const double sg = loc[k] >= 0.0 ? 1.0 : -1.0;
        cl[k] = sg * B.h[k];
        nb = scl(B.u[k], sg);
        gap = -pen - r;
    }
    pt = at(B, cl[0], cl[1], cl[2]);
    normal = scl(nb, -1.0);
    return gap <= margin;
}

// separation along the unit axis L: |T.L| minus both boxes' half widths
OVL_HD double axis_sep(const Obb &A, const Obb &B, double3 T, double3 L) {
    double s = fabs(dot(T, L));
    for (int k = 0; k < 3; ++k) s -= A.h[k] * fabs(dot(A.u[k], L)) + B.h[k] * fabs(dot(B.u[k], L));
    return s;
}

// keep the part of polygon P (n points) with dot(x, e) <= off (convex clip)
OVL_HD int clip_half(const double3 *P, int n, double3 e, double off, double3 *Q) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double3 a = P[i], b = P[i + 1 == n ? 0 : i + 1];
        const double da = dot(a, e) - off, db = dot(b, e) - off;
        if (da <= 0.0) Q[m++] = a;
        if ((da <= 0.0) != (db <= 0.0)) Q[m++] = add(a, scl(sub(b, a), da / (da - db)));
    }
    return m;
}

// Box A (first) against box B (second).  Returns the count (0 when an axis
// separates them by more than the margin; axis = -1 then).  normal: A -> B.
OVL_HD int box_box(const Obb &A, const Obb &B, double margin, double3 pts[4], double gaps[4], double3 &normal,
                   int &axis, double &sep) {
    axis = -1;
    const double3 T = sub(B.c, A.c);
    double3 L[15];
    double s[15];
    bool ok[15];
    for (int k = 0; k < 3; ++k) {
        L[k] = A.u[k];
        L[3 + k] = B.u[k];
        ok[k] = ok[3 + k] = true;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const int k = 6 + 3 * i + j;
            const double3 x = crs(A.u[i], B.u[j]);
            const double len = sqrt(dot(x, x));
            ok[k] = len > kEdgeMin;
            L[k] = ok[k] ? scl(x, 1.0 / len) : d3(0.0, 0.0, 0.0);
        }
    for (int k = 0; k < 15; ++k) {
        s[k] = ok[k] ? axis_sep(A, B, T, L[k]) : -INFINITY;
        if (s[k] > margin) return 0;
    }
    int face = 0, edge = -1;
    for (int k = 1; k < 6; ++k)
        if (s[k] > s[face] + kTieLen) face = k;
    for (int k = 6; k < 15; ++k)
        if (ok[k] && (edge < 0 || s[k] > s[edge] + kTieLen)) edge = k;
    double hmin = A.h[0];
    for (int k = 0; k < 3; ++k) hmin = fmin(hmin, fmin(A.h[k], B.h[k]));
    const double edge_thr = s[face] + 0.05 * fabs(s[face]) + 0.01 * hmin;
    const int best = (edge >= 0 && s[edge] > edge_thr) ? edge : face;
    axis = best;
    sep = s[best];
    normal = dot(T, L[best]) < 0.0 ? scl(L[best], -1.0) : L[best];

    if (best >= 6) {
        // the two supporting edges: A's along a_i nearest B, B's along b_j nearest A
        const int i = (best - 6) / 3, j = (best - 6) % 3;
        double3 pa = A.c, pb = B.c;
        for (int k = 0; k < 3; ++k) {
            if (k != i) pa = add(pa, scl(A.u[k], dot(A.u[k], normal) >= 0.0 ? A.h[k] : -A.h[k]));
            if (k != j) pb = add(pb, scl(B.u[k], dot(B.u[k], normal) <= 0.0 ? B.h[k] : -B.h[k]));
        }
        // nearest points of pa + t a_i (|t| <= h) and pb + v b_j (|v| <= h)
        const double3 w = sub(pa, pb);
        const double c = dot(A.u[i], B.u[j]), e = dot(A.u[i], w), f = dot(B.u[j], w);
        const double den = 1.0 - c * c;                 // >= kEdgeMin^2 on an edge axis
        double t = (c * f - e) / den;
        t = fmin(fmax(t, -A.h[i]), A.h[i]);
        const double v = fmin(fmax(c * t + f, -B.h[j]), B.h[j]);
        t = fmin(fmax(c * v - e, -A.h[i]), A.h[i]);
        pts[0] = scl(add(add(pa, scl(A.u[i], t)), add(pb, scl(B.u[j], v))), 0.5);
        gaps[0] = sep;
        return 1;
    }

    // face axis: the owner is the reference box, the other the incident one
    const bool refA = best < 3;
    const Obb &R = refA ? A : B, &I = refA ? B : A;
    const int f = best % 3;
    const double3 nr = refA ? normal : scl(normal, -1.0);   // reference face normal, towards I
    int fi = 0;
    double most = fabs(dot(I.u[0], nr));
    for (int k = 1; k < 3; ++k) {
        const double d = fabs(dot(I.u[k], nr));
        if (d > most + kTieDir) { most = d; fi = k; }
    }
    const double si = dot(I.u[fi], nr) > 0.0 ? -1.0 : 1.0;
    const int a1 = fi == 0 ? 1 : 0, a2 = fi == 2 ? 1 : 2;
    double3 poly[16], tmp[16];
    const double3 fc = add(I.c, scl(I.u[fi], si * I.h[fi]));
    const double su[4] = {-1.0, 1.0, 1.0, -1.0}, sv[4] = {-1.0, -1.0, 1.0, 1.0};
    for (int k = 0; k < 4; ++k)
        poly[k] = add(fc, add(scl(I.u[a1], su[k] * I.h[a1]), scl(I.u[a2], sv[k] * I.h[a2])));
    int m = 4;
    const int r1 = f == 0 ? 1 : 0, r2 = f == 2 ? 1 : 2;
    const int side[2] = {r1, r2};
    for (int t = 0; t < 2 && m > 0; ++t) {
        const double3 e = R.u[side[t]];
        m = clip_half(poly, m, e, dot(R.c, e) + R.h[side[t]] + kTieLen, tmp);
        if (m > 0) m = clip_half(tmp, m, scl(e, -1.0), -dot(R.c, e) + R.h[side[t]] + kTieLen, poly);
    }
    const double3 rc = add(R.c, scl(nr, R.h[f]));         // reference face centre
    double3 P[16];
    double G[16];
    int kept = 0;
    for (int k = 0; k < m; ++k) {
        const double g = dot(sub(poly[k], rc), nr);
        if (g <= margin) { P[kept] = poly[k]; G[kept] = g; ++kept; }
    }
    kept = keep_deepest(P, G, kept, 4);
    for (int k = 0; k < kept; ++k) { pts[k] = P[k]; gaps[k] = G[k]; }
    return kept;
}

// ---- bounding tests (the step's FP32 contact decisions for spheres) -------
// two spheres (or bounding spheres): ((dx dx + dy dy) + dz dz) <= ((ra + rb) + margin)^2
OVL_HD bool spheres_touch(float3 a, float3 b, float ra, float rb, float margin) {
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    const float d2 = (dx * dx + dy * dy) + dz * dz;
    const float rs = (ra + rb) + margin;
    return d2 <= rs * rs;
}

// a sphere (or bounding sphere) and the plane n.x = d: ((n.p) - d) - r <= margin
OVL_HD bool sphere_plane_touch(float3 c, float r, float4 pl, float margin) {
    const float dotp = (pl.x * c.x + pl.y * c.y) + pl.z * c.z;
    return (dotp - pl.w) - r <= margin;
}

// ---- box rows ------------------------------------------------------------
// world inverse inertia of a solid box (inverse mass im, half extents h):
// R diag(1 / I_k) R^T, I_k = m/3 (h_j^2 + h_l^2); row-major 3 x 3
OVL_HD void inv_inertia_world(const Obb &B, float im, float Iw[9]) {
    float d[3];
    for (int k = 0; k < 3; ++k) {
        const float a = (float)B.h[(k + 1) % 3], b = (float)B.h[(k + 2) % 3];
        d[k] = im > 0.f ? 3.f * im / (a * a + b * b) : 0.f;
    }
    const float3 u0 = to_f(B.u[0]), u1 = to_f(B.u[1]), u2 = to_f(B.u[2]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Iw[3 * r + c] = comp(u0, r) * d[0] * comp(u0, c) + comp(u1, r) * d[1] * comp(u1, c) +
                            comp(u2, r) * d[2] * comp(u2, c);
}

OVL_HD float3 mul(const float Iw[9], float3 v) {
    return v3(Iw[0] * v.x + Iw[1] * v.y + Iw[2] * v.z, Iw[3] * v.x + Iw[4] * v.y + Iw[5] * v.z,
              Iw[6] * v.x + Iw[7] * v.y + Iw[8] * v.z);
}

// One constraint row of the first body against a static second one: along
// direction d at lever r, w = -d.v - (r x d).omega; the row keeps r x d,
// Iw^-1 (r x d) and k = 1 / (1/m + (r x d).Iw^-1 (r x d)).
struct Row1 {
    float3 d, rxd, irxd;
    float k, target;
};

OVL_HD Row1 make_row(float3 d, float3 r, float im, const float Iw[9], float target) {
    Row1 row;
    row.d = d;
    row.rxd = crs(r, d);
    row.irxd = mul(Iw, row.rxd);
    row.k = 1.f / (im + dot(row.rxd, row.irxd));
    row.target = target;
    return row;
}

// clamp by comparisons: unlike fminf/fmaxf, the result at signed-zero ties
// (a bound of -0 against +0) is the same on host and device
OVL_HD float clampf(float x, float lo, float hi) { return x < lo ? lo : (x > hi ? hi : x); }

// projected Gauss-Seidel update of one row: the body takes -d (l' - l)
OVL_HD void solve_row(const Row1 &row, float lo, float hi, float im, float3 &v, float3 &w, float &lam) {
    const float wv = -dot(row.d, v) - dot(row.rxd, w);
    const float ln = clampf(lam + row.k * (row.target - wv), lo, hi);
    const float dl = ln - lam;
    lam = ln;
    v = sub(v, scl(row.d, im * dl));
    w = sub(w, scl(row.irxd, dl));
}

// tangent t1 of a contact normal: normalise(e_k - n_k n) for the axis k of
// the smallest |n_k|, a later axis winning only by more than kTieDir
OVL_HD float3 tangent1(float3 n) {
    const float tie = (float)kTieDir;
    int k = 0;
    float m = fabsf(n.x);
    if (fabsf(n.y) < m - tie) { m = fabsf(n.y); k = 1; }
    if (fabsf(n.z) < m - tie) k = 2;
    const float nk = comp(n, k);
    float3 t = scl(n, -nk);
    if (k == 0) t.x += 1.f; else if (k == 1) t.y += 1.f; else t.z += 1.f;
    return scl(t, 1.f / sqrtf(dot(t, t)));
}

// One velocity step of a single box (first) on a static plane (second):
// gravity, then `iters` sweeps over (normal, t1, t2) of every box_plane
// contact in order.  Normal bounds [0, inf) with target -phi/dt when phi > 0
// else erp max(-phi - slop, 0)/dt; tangents within +-mu lambda_n.
// lam[12]: (n, t1, t2) per contact.  Returns the contact count.
OVL_HD int box_plane_step(const Obb &B, float im, float4 plane, float mu, float dt, float3 g, float erp,
                          float slop, float margin, int iters, float3 &v, float3 &w, float lam[12]) {
    float3 pts[4], n;
    float gaps[4], Iw[9];
    double3 pd[4], nd;
    double gd[4];
    const int m = box_plane(B, plane, margin, pd, gd, nd);
    for (int i = 0; i < m; ++i) { pts[i] = to_f(pd[i]); gaps[i] = (float)gd[i]; }
    n = to_f(nd);
    inv_inertia_world(B, im, Iw);
    v = add(v, scl(g, dt));
    const float3 t1 = tangent1(n), t2 = crs(n, t1);
    Row1 rows[12];
    for (int c = 0; c < m; ++c) {
        const float3 r = sub(pts[c], to_f(B.c));
        const float pen = -gaps[c] - slop;
        const float tn = gaps[c] > 0.f ? -gaps[c] / dt : erp * (pen > 0.f ? pen : 0.f) / dt;
        rows[3 * c] = make_row(n, r, im, Iw, tn);
        rows[3 * c + 1] = make_row(t1, r, im, Iw, 0.f);
        rows[3 * c + 2] = make_row(t2, r, im, Iw, 0.f);
        lam[3 * c] = lam[3 * c + 1] = lam[3 * c + 2] = 0.f;
    }
    for (int it = 0; it < iters; ++it)
        for (int c = 0; c < m; ++c) {
            solve_row(rows[3 * c], 0.f, INFINITY, im, v, w, lam[3 * c]);
            const float lim = mu * lam[3 * c];
            solve_row(rows[3 * c + 1], -lim, lim, im, v, w, lam[3 * c + 1]);
            solve_row(rows[3 * c + 2], -lim, lim, im, v, w, lam[3 * c + 2]);
        }
    return m;
}

#undef OVL_HD

}  // namespace box
}  // namespace ovl
