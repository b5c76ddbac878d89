/* box_oracle.c -- TEST INFRASTRUCTURE ONLY (the CUDA library never links,
 * includes or calls it).  Plain FP64 reference geometry for box contacts,
 * the shapes of the paper's Building and Bridge scenes (Section 6: floors,
 * walls, columns and planks), written from the textbook definitions:
 *
 *   box_plane   the box's vertices within the margin of a plane, at most
 *               the 4 deepest
 *   sphere_box  the point of the box closest to the sphere's centre (or,
 *               with the centre inside, its projection on the face of least
 *               penetration)
 *   box_box     the separating-axis test for two oriented boxes over their
 *               15 candidate axes (3 + 3 face normals, 9 edge cross
 *               products); on a face axis the incident face clipped against
 *               the reference face's side planes (Sutherland-Hodgman),
 *               keeping the 4 deepest points; on an edge axis one point
 *               between the two supporting edges
 *
 * Conventions (shared with the sphere contacts of ovl_oracle.c): the normal
 * points from the first shape towards the second; the gap is positive when
 * they are apart and negative when they overlap; a contact exists when the
 * gap is <= margin.  Quaternions are (w, x, y, z) and unit; a box is a
 * centre, an orientation and three half extents.
 *
 * Readings (the paper gives no box geometry; its engine supplies it):
 *  - contact point: a box vertex (box-plane), the box surface point
 *    (sphere-box), the clipped incident-face point (box-box, face axis), the
 *    midpoint of the closest points of the two edges (box-box, edge axis);
 *  - an edge axis is chosen over the best face axis only when its
 *    separation exceeds the face separation by more than 5 % of its
 *    magnitude + 0.01 x the smallest half extent (faces give stable 4-point
 *    manifolds; near-ties go to them, separated or penetrating);
 *  - decisions with a tolerance, so that a computation in any precision
 *    that is accurate to well under the tolerance decides alike (exactly
 *    aligned boxes, as in a building, tie in exact arithmetic):
 *      axes: scanning A's faces, B's faces, then a_i x b_j (i major), a
 *        later axis replaces the best so far only if its separation exceeds
 *        it by more than ORC_BOX_TIE_LEN (0.3 mm); an a_i x b_j axis exists
 *        only when |a_i x b_j| > ORC_BOX_EDGE_MIN;
 *      the incident face: the most anti-parallel face, a later one winning
 *        only by more than ORC_BOX_TIE_DIR in |cosine|;
 *      the least-penetrated face of a box holding a sphere's centre: a later
 *        face wins only by more than ORC_BOX_TIE_LEN;
 *      clipping keeps the points within ORC_BOX_TIE_LEN outside a side plane
 *        of the reference face (it clips at that distance);
 *      the 4 deepest: a selection that takes, in candidate order, the first
 *        candidate not deeper than the deepest remaining one by more than
 *        ORC_BOX_TIE_LEN;
 *  - every decision reports how close its quantity came to the threshold, in
 *    units of a band (ORC_BOX_BAND_LEN for lengths, ORC_BOX_BAND_DIR for
 *    cosines): *amb receives the smallest such distance.  amb < 1 marks a
 *    pair whose decisions an FP32 computation may take differently. */
#define ORC_BOX_TIE_LEN 3e-4
#define ORC_BOX_TIE_DIR 1e-4
#define ORC_BOX_EDGE_MIN 1e-3
#define ORC_BOX_BAND_LEN 3e-5
#define ORC_BOX_BAND_DIR 1e-5
#include <math.h>
#include <string.h>

/* distance of x from a decision threshold, in bands, into *amb */
static void note(double *amb, double x, double thr, double band) {
    const double d = fabs(x - thr) / band;
    if (amb && d < *amb) *amb = d;
}

static void quat_R(const double q[4], double R[9]) {
    /* R[3 r + c]; column k is the box's axis k in world coordinates */
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void axis_of(const double R[9], int k, double out[3]) {
    out[0] = R[k]; out[1] = R[3 + k]; out[2] = R[6 + k];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* keep the k deepest of m candidates: k times, among the remaining
 * candidates in their order, the first one whose gap is not more than
 * ORC_BOX_TIE_LEN above the smallest remaining gap; pts/gaps are compacted
 * in place in that order; returns the kept count */
static int keep_deepest(double *pts, double *gaps, int m, int k, double *amb) {
    int order[16];
    for (int i = 0; i < m; ++i) order[i] = i;
    const int n = m < k ? m : k;
    for (int i = 0; i < n; ++i) {
        double gmin = gaps[order[i]];
        for (int j = i + 1; j < m; ++j)
            if (gaps[order[j]] < gmin) gmin = gaps[order[j]];
        int pick = i;
        for (int j = i; j < m; ++j) {
            note(amb, gaps[order[j]], gmin + ORC_BOX_TIE_LEN, ORC_BOX_BAND_LEN);
            if (gaps[order[j]] <= gmin + ORC_BOX_TIE_LEN) { pick = j; break; }
        }
        const int o = order[pick];
        for (int j = pick; j > i; --j) order[j] = order[j - 1];
        order[i] = o;
    }
    double p2[48], g2[16];
    for (int i = 0; i < n; ++i) {
        memcpy(p2 + 3 * i, pts + 3 * order[i], 3 * sizeof(double));
        g2[i] = gaps[order[i]];
    }
    memcpy(pts, p2, (size_t)n * 3 * sizeof(double));
    memcpy(gaps, g2, (size_t)n * sizeof(double));
    return n;
}

/* Box (first) against the plane {x : n.x = d} (second; n unit, pointing out
 * of the solid).  pts[4][3], gaps[4]; normal[3] = -n.  Returns the count. */
int box_plane(const double c[3], const double q[4], const double h[3], const double plane[4],
              double margin, double pts[12], double gaps[4], double normal[3], double *amb) {
    double R[9], P[24], G[8];
    quat_R(q, R);
    int m = 0;
    for (int v = 0; v < 8; ++v) {
        const double s[3] = {(v & 1) ? 1.0 : -1.0, (v & 2) ? 1.0 : -1.0, (v & 4) ? 1.0 : -1.0};
        double p[3];
        for (int r = 0; r < 3; ++r)
            p[r] = c[r] + R[3 * r] * s[0] * h[0] + R[3 * r + 1] * s[1] * h[1] + R[3 * r + 2] * s[2] * h[2];
        const double g = plane[0] * p[0] + plane[1] * p[1] + plane[2] * p[2] - plane[3];
        note(amb, g, margin, ORC_BOX_BAND_LEN);
        if (g <= margin) {
            memcpy(P + 3 * m, p, sizeof p);
            G[m++] = g;
        }
    }
    m = keep_deepest(P, G, m, 4, amb);
    memcpy(pts, P, (size_t)m * 3 * sizeof(double));
    memcpy(gaps, G, (size_t)m * sizeof(double));
    normal[0] = -plane[0]; normal[1] = -plane[1]; normal[2] = -plane[2];
    return m;
}

/* Sphere (first: centre s, radius r) against a box (second).  One contact:
 * pt[3] on the box surface, normal[3] from the sphere towards the box,
 * *gap.  Returns 1 when gap <= margin, else 0 (outputs still written). */
int sphere_box(const double s[3], double r, const double c[3], const double q[4], const double h[3],
               double margin, double pt[3], double normal[3], double *gap, double *amb) {
    double R[9], p[3], cl[3], nb[3];
    quat_R(q, R);
    const double d[3] = {s[0] - c[0], s[1] - c[1], s[2] - c[2]};
    for (int k = 0; k < 3; ++k) p[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];   /* box frame */
    int inside = 1;
    for (int k = 0; k < 3; ++k) {
        cl[k] = p[k] < -h[k] ? -h[k] : (p[k] > h[k] ? h[k] : p[k]);
        note(amb, fabs(p[k]), h[k], ORC_BOX_BAND_LEN);
        if (cl[k] != p[k]) inside = 0;
    }
    if (!inside) {
        const double e[3] = {p[0] - cl[0], p[1] - cl[1], p[2] - cl[2]};
        const double dist = sqrt(dot3(e, e));
        for (int k = 0; k < 3; ++k) nb[k] = e[k] / dist;              /* box -> sphere */
        *gap = dist - r;
    } else {
        int kk = 0;
        double pen = h[0] - fabs(p[0]);
        for (int k = 1; k < 3; ++k) {
            note(amb, h[k] - fabs(p[k]), pen - ORC_BOX_TIE_LEN, ORC_BOX_BAND_LEN);
            if (h[k] - fabs(p[k]) < pen - ORC_BOX_TIE_LEN) { pen = h[k] - fabs(p[k]); kk = k; }
        }
        note(amb, p[kk], 0.0, ORC_BOX_BAND_LEN);
        const double sg = p[kk] >= 0 ? 1.0 : -1.0;
        nb[0] = nb[1] = nb[2] = 0.0;
        nb[kk] = sg;
        cl[kk] = sg * h[kk];                                        /* projection on that face */
        *gap = -pen - r;
    }
    for (int r3 = 0; r3 < 3; ++r3) {
        pt[r3] = c[r3] + R[3 * r3] * cl[0] + R[3 * r3 + 1] * cl[1] + R[3 * r3 + 2] * cl[2];
        normal[r3] = -(R[3 * r3] * nb[0] + R[3 * r3 + 1] * nb[1] + R[3 * r3 + 2] * nb[2]);
    }
    note(amb, *gap, margin, ORC_BOX_BAND_LEN);
    return *gap <= margin;
}

/* separation of two boxes along the unit axis L: |T.L| - (A's and B's
 * half projections); positive = a gap along L */
static double separation(const double T[3], const double L[3], const double RA[9], const double hA[3],
                         const double RB[9], const double hB[3]) {
    double s = fabs(dot3(T, L)), ax[3];
    for (int k = 0; k < 3; ++k) {
        axis_of(RA, k, ax);
        s -= hA[k] * fabs(dot3(ax, L));
        axis_of(RB, k, ax);
        s -= hB[k] * fabs(dot3(ax, L));
    }
    return s;
}

/* Sutherland-Hodgman: clip polygon P (n points) by {x : dot(x, e) <= off}
 * (the caller widens off by ORC_BOX_TIE_LEN); returns the new count (at most
 * n + 1 per plane, <= 8 here) */
static int clip_plane(const double *P, int n, const double e[3], double off, double *out, double *amb) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double *a = P + 3 * i, *b = P + 3 * ((i + 1) % n);
        const double da = dot3(a, e) - off, db = dot3(b, e) - off;
        note(amb, da, 0.0, ORC_BOX_BAND_LEN);
        if (da <= 0) { memcpy(out + 3 * m, a, 3 * sizeof(double)); ++m; }
        if ((da <= 0) != (db <= 0)) {
            const double t = da / (da - db);
            for (int k = 0; k < 3; ++k) out[3 * m + k] = a[k] + t * (b[k] - a[k]);
            ++m;
        }
    }
    return m;
}

/* Box A (first) against box B (second).  Up to 4 contacts: pts[4][3],
 * gaps[4], one normal[3] from A towards B; *axis receives the chosen axis
 * (0-2 A's faces, 3-5 B's faces, 6 + 3 i + j for a_i x b_j) and *sep its
 * separation.  Returns the count (0 when some axis separates them by more
 * than the margin). */
int box_box(const double cA[3], const double qA[4], const double hA[3], const double cB[3],
            const double qB[4], const double hB[3], double margin, double pts[12], double gaps[4],
            double normal[3], int *axis, double *sep, double *amb) {
    double RA[9], RB[9];
    quat_R(qA, RA);
    quat_R(qB, RB);
    const double T[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};
    double L[15][3];
    int valid[15];
    double s[15];
    for (int k = 0; k < 3; ++k) {
        axis_of(RA, k, L[k]);
        axis_of(RB, k, L[3 + k]);
        valid[k] = valid[3 + k] = 1;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a[3], b[3], x[3];
            axis_of(RA, i, a);
            axis_of(RB, j, b);
            cross3(a, b, x);
            const double len = sqrt(dot3(x, x));
            const int k = 6 + 3 * i + j;
            note(amb, len, ORC_BOX_EDGE_MIN, ORC_BOX_BAND_DIR);
            valid[k] = len > ORC_BOX_EDGE_MIN;             /* near-parallel edges: the faces cover them */
            for (int r = 0; r < 3; ++r) L[k][r] = valid[k] ? x[r] / len : 0.0;
        }
    for (int k = 0; k < 15; ++k) {
        s[k] = valid[k] ? separation(T, L[k], RA, hA, RB, hB) : -INFINITY;
        if (valid[k]) note(amb, s[k], margin, ORC_BOX_BAND_LEN);
        if (valid[k] && s[k] > margin) return 0;
    }
    int bf = 0, be = -1;
    for (int k = 1; k < 6; ++k) {
        note(amb, s[k], s[bf] + ORC_BOX_TIE_LEN, ORC_BOX_BAND_LEN);
        if (s[k] > s[bf] + ORC_BOX_TIE_LEN) bf = k;
    }
    for (int k = 6; k < 15; ++k) {
        if (!valid[k]) continue;
        if (be >= 0) note(amb, s[k], s[be] + ORC_BOX_TIE_LEN, ORC_BOX_BAND_LEN);
        if (be < 0 || s[k] > s[be] + ORC_BOX_TIE_LEN) be = k;
    }
    double hmin = hA[0];
    for (int k = 0; k < 3; ++k) {
        if (hA[k] < hmin) hmin = hA[k];
        if (hB[k] < hmin) hmin = hB[k];
    }
    const double edge_thr = s[bf] + 0.05 * fabs(s[bf]) + 0.01 * hmin;
    if (be >= 0) note(amb, s[be], edge_thr, ORC_BOX_BAND_LEN);
    const int best = (be >= 0 && s[be] > edge_thr) ? be : bf;
    *axis = best;
    *sep = s[best];
    note(amb, dot3(T, L[best]), 0.0, ORC_BOX_BAND_LEN);
    const double sgn = dot3(T, L[best]) < 0 ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r) normal[r] = sgn * L[best][r];     /* A -> B */

    if (best >= 6) {
        /* supporting edge of A along a_i (towards B) and of B along b_j (towards A) */
        const int i = (best - 6) / 3, j = (best - 6) % 3;
        double pA[3], pB[3], ai[3], bj[3], ax[3];
        memcpy(pA, cA, sizeof pA);
        memcpy(pB, cB, sizeof pB);
        for (int k = 0; k < 3; ++k) {
            if (k != i) {
                axis_of(RA, k, ax);
                note(amb, dot3(ax, normal), 0.0, ORC_BOX_BAND_DIR);
                const double sg = dot3(ax, normal) >= 0 ? 1.0 : -1.0;
                for (int r = 0; r < 3; ++r) pA[r] += sg * hA[k] * ax[r];
            }
            if (k != j) {
                axis_of(RB, k, ax);
                note(amb, dot3(ax, normal), 0.0, ORC_BOX_BAND_DIR);
                const double sg = dot3(ax, normal) <= 0 ? 1.0 : -1.0;
                for (int r = 0; r < 3; ++r) pB[r] += sg * hB[k] * ax[r];
            }
        }
        axis_of(RA, i, ai);
        axis_of(RB, j, bj);
        /* closest points of the segments pA + u ai (|u| <= hA_i), pB + v bj */
        const double w0[3] = {pA[0] - pB[0], pA[1] - pB[1], pA[2] - pB[2]};
        const double b = dot3(ai, bj), cc = dot3(ai, w0), f = dot3(bj, w0);
        const double den = 1.0 - b * b;
        double u = (b * f - cc) / den;                     /* den >= ORC_BOX_EDGE_MIN^2 on an edge axis */
        u = u < -hA[i] ? -hA[i] : (u > hA[i] ? hA[i] : u);
        double v = b * u + f;
        v = v < -hB[j] ? -hB[j] : (v > hB[j] ? hB[j] : v);
        u = b * v - cc;
        u = u < -hA[i] ? -hA[i] : (u > hA[i] ? hA[i] : u);
        for (int r = 0; r < 3; ++r) pts[r] = 0.5 * ((pA[r] + u * ai[r]) + (pB[r] + v * bj[r]));
        gaps[0] = s[best];
        return 1;
    }

    /* face axis: reference box (owns the axis), incident box (the other) */
    const int refA = best < 3;
    const int f = best % 3;
    const double *Rr = refA ? RA : RB, *Ri = refA ? RB : RA;
    const double *hr = refA ? hA : hB, *hi = refA ? hB : hA;
    const double *cr = refA ? cA : cB, *ci = refA ? cB : cA;
    double nref[3];                                     /* reference face normal, towards the incident box */
    for (int r = 0; r < 3; ++r) nref[r] = refA ? normal[r] : -normal[r];
    /* incident face: the face of the incident box most anti-parallel to nref */
    int fi = 0;
    double best_d = -1.0, ax[3];
    for (int k = 0; k < 3; ++k) {
        axis_of(Ri, k, ax);
        const double d = fabs(dot3(ax, nref));
        if (k > 0) note(amb, d, best_d + ORC_BOX_TIE_DIR, ORC_BOX_BAND_DIR);
        if (k == 0 || d > best_d + ORC_BOX_TIE_DIR) { best_d = d; fi = k; }
    }
    axis_of(Ri, fi, ax);
    const double si = dot3(ax, nref) > 0 ? -1.0 : 1.0;
    const int u = fi == 0 ? 1 : 0, v = fi == 2 ? 1 : 2;
    double eu[3], ev[3], poly[3 * 16], tmp[3 * 16];
    axis_of(Ri, u, eu);
    axis_of(Ri, v, ev);
    const double cu[4] = {-1, 1, 1, -1}, cv[4] = {-1, -1, 1, 1};
    for (int k = 0; k < 4; ++k)
        for (int r = 0; r < 3; ++r)
            poly[3 * k + r] = ci[r] + si * hi[fi] * ax[r] + cu[k] * hi[u] * eu[r] + cv[k] * hi[v] * ev[r];
    int m = 4;
    /* side planes of the reference face: |(x - cr).e| <= hr for its two in-plane axes */
    const int ru = f == 0 ? 1 : 0, rv = f == 2 ? 1 : 2;
    const int sides[2] = {ru, rv};
    for (int t = 0; t < 2 && m > 0; ++t) {
        double e[3], ne[3];
        axis_of(Rr, sides[t], e);
        for (int r = 0; r < 3; ++r) ne[r] = -e[r];
        m = clip_plane(poly, m, e, dot3(cr, e) + hr[sides[t]] + ORC_BOX_TIE_LEN, tmp, amb);
        if (m == 0) break;
        m = clip_plane(tmp, m, ne, dot3(cr, ne) + hr[sides[t]] + ORC_BOX_TIE_LEN, poly, amb);
    }
    /* depth of each point below the reference face */
    double fc[3], P[3 * 16], G[16];
    for (int r = 0; r < 3; ++r) fc[r] = cr[r] + hr[f] * nref[r];
    int kept = 0;
    for (int k = 0; k < m; ++k) {
        const double d[3] = {poly[3 * k] - fc[0], poly[3 * k + 1] - fc[1], poly[3 * k + 2] - fc[2]};
        const double g = dot3(d, nref);
        note(amb, g, margin, ORC_BOX_BAND_LEN);
        if (g <= margin) {
            memcpy(P + 3 * kept, poly + 3 * k, 3 * sizeof(double));
            G[kept++] = g;
        }
    }
    kept = keep_deepest(P, G, kept, 4, amb);
    memcpy(pts, P, (size_t)kept * 3 * sizeof(double));
    memcpy(gaps, G, (size_t)kept * sizeof(double));
    return kept;
}

/* the separations of A and B along all 15 candidate axes, in box_box's
 * order (-inf for a parallel-edge pair, which has no axis) */
void box_box_axes(const double cA[3], const double qA[4], const double hA[3], const double cB[3],
                  const double qB[4], const double hB[3], double s[15]) {
    double RA[9], RB[9], L[3], a[3], b[3];
    quat_R(qA, RA);
    quat_R(qB, RB);
    const double T[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};
    for (int k = 0; k < 3; ++k) {
        axis_of(RA, k, L);
        s[k] = separation(T, L, RA, hA, RB, hB);
        axis_of(RB, k, L);
        s[3 + k] = separation(T, L, RA, hA, RB, hB);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            axis_of(RA, i, a);
            axis_of(RB, j, b);
            cross3(a, b, L);
            const double len = sqrt(dot3(L, L));
            if (len > ORC_BOX_EDGE_MIN) {
                for (int r = 0; r < 3; ++r) L[r] /= len;
                s[6 + 3 * i + j] = separation(T, L, RA, hA, RB, hB);
            } else {
                s[6 + 3 * i + j] = -INFINITY;
            }
        }
}

/* ---- box rows ------------------------------------------------------------
 * World inverse inertia of a solid box of inverse mass inv_mass and half
 * extents h: R diag(1 / I_k) R^T with I_k = m/3 (h_j^2 + h_l^2) (j, l the
 * other two axes).  Iw row-major. */
void box_inv_inertia_world(const double q[4], const double h[3], double inv_mass, double Iw[9]) {
    double R[9], d[3];
    quat_R(q, R);
    for (int k = 0; k < 3; ++k) {
        const double a = h[(k + 1) % 3], b = h[(k + 2) % 3];
        d[k] = inv_mass > 0 ? 3.0 * inv_mass / (a * a + b * b) : 0.0;   /* 1 / I_k */
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Iw[3 * r + c] = R[3 * r] * d[0] * R[3 * c] + R[3 * r + 1] * d[1] * R[3 * c + 1] +
                            R[3 * r + 2] * d[2] * R[3 * c + 2];
}

static void mat3_vec(const double M[9], const double v[3], double o[3]) {
    for (int r = 0; r < 3; ++r) o[r] = M[3 * r] * v[0] + M[3 * r + 1] * v[1] + M[3 * r + 2] * v[2];
}

/* One velocity step (Algorithm 1's solve, Eq 1-7) of a single dynamic box
 * (first body) against a static plane (second): v += dt g, then `iters`
 * Gauss-Seidel sweeps over the rows of the box_plane contacts, in their
 * order, each as normal, t1, t2.  Row d at lever r (contact point minus the
 * centre): w = -d.v - (r x d).omega, k = 1 / (1/m + (r x d).Iw^-1 (r x d)),
 * lambda' = clamp(lambda + k (target - w)), and the box takes the impulse
 * -d (lambda' - lambda).  Normal bounds [0, inf), target -phi/dt when phi >
 * 0 else erp max(-phi - slop, 0)/dt; tangents bounded by +-mu lambda_n
 * (current), t1 = normalise(e_k - n_k n) for the axis k of the smallest
 * |n_k| (ties to the lower index), t2 = n x t1.  v[3], w[3] in/out;
 * lam[12] = (n, t1, t2) impulses per contact.  Returns the contact count. */
int box_plane_step(const double x[3], const double q[4], const double h[3], double inv_mass,
                   const double plane[4], double mu, double dt, const double g[3], double erp, double slop,
                   double margin, int iters, double v[3], double w[3], double lam[12]) {
    double pts[12], gaps[4], n[3], Iw[9];
    const int m = box_plane(x, q, h, plane, margin, pts, gaps, n, NULL);
    box_inv_inertia_world(q, h, inv_mass, Iw);
    for (int k = 0; k < 3; ++k) v[k] += dt * g[k];
    /* tangent axis of the normal */
    int ka = 0;
    double mn = fabs(n[0]);
    for (int k = 1; k < 3; ++k)
        if (fabs(n[k]) < mn) { mn = fabs(n[k]); ka = k; }
    double t1[3] = {-n[ka] * n[0], -n[ka] * n[1], -n[ka] * n[2]}, t2[3];
    t1[ka] += 1.0;
    const double l1 = sqrt(dot3(t1, t1));
    for (int k = 0; k < 3; ++k) t1[k] /= l1;
    cross3(n, t1, t2);
    const double *dirs[3] = {n, t1, t2};
    double rxd[12][3], Irxd[12][3], kk[12], tgt[12];
    for (int c = 0; c < m; ++c) {
        const double r[3] = {pts[3 * c] - x[0], pts[3 * c + 1] - x[1], pts[3 * c + 2] - x[2]};
        for (int j = 0; j < 3; ++j) {
            const int i = 3 * c + j;
            cross3(r, dirs[j], rxd[i]);
            mat3_vec(Iw, rxd[i], Irxd[i]);
            kk[i] = 1.0 / (inv_mass + dot3(rxd[i], Irxd[i]));
            tgt[i] = 0.0;
            lam[i] = 0.0;
        }
        tgt[3 * c] = gaps[c] > 0 ? -gaps[c] / dt : erp * fmax(-gaps[c] - slop, 0.0) / dt;
    }
    for (int it = 0; it < iters; ++it)
        for (int c = 0; c < m; ++c)
            for (int j = 0; j < 3; ++j) {
                const int i = 3 * c + j;
                const double wv = -dot3(dirs[j], v) - dot3(rxd[i], w);
                double lo = 0.0, hi = INFINITY;
                if (j > 0) { hi = mu * lam[3 * c]; lo = -hi; }
                double ln = lam[i] + kk[i] * (tgt[i] - wv);
                ln = ln < lo ? lo : (ln > hi ? hi : ln);
                const double dl = ln - lam[i];
                lam[i] = ln;
                for (int k = 0; k < 3; ++k) {
                    v[k] -= inv_mass * dirs[j][k] * dl;
                    w[k] -= Irxd[i][k] * dl;
                }
            }
    return m;
}
