/*
 * ovl_oracle.c -- plain, slow FP64 CPU oracle for one timestep of the
 * overlapping-partition rigid-body method of Kale & Kry, "Distributed
 * Simulation of Large Multi-body Systems" (Algorithm 1, Sections 3-5).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, calls or
 * executes this file: it is used by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg.  It shares no code, header, table or constant
 * generator with the CUDA library; both are fed from the seeded scene
 * generators only.
 *
 * Every step is written in the paper's order and notation, with no blocking,
 * fusion or reordering.  Three loops whose iterations are independent -- the
 * contacts of each body, the solve of each worker (workers share nothing
 * during a step, Section 4) and the search of D(o, i) from each overlap body
 * -- may run on several threads (orc_set_threads; default 1); each
 * iteration's arithmetic is the same, so no result depends on the thread
 * count:
 *
 *   contacts  (Alg 1 contact generation, Section 5.4)      orc_contacts
 *   graph G^t (Section 5.1, constraint graph)              orc_graph
 *   LOADBALANCE (Alg 6) + BRIDGE (Alg 7)                   orc_load_balance
 *   ASSIGNTOOVERLAPSET (Alg 2) + GROWOVERLAP (Alg 3)       orc_assign_overlap
 *   P_i, O (Eq 9, Eq 10)                                   entries / pairs
 *   per-worker PGS on the MLCP of Eq 1-7 + integration     solve_worker
 *   D(o,i) (Eq 16, searched as in Alg 5)                   orc_geodesics
 *   weights (Eq 15) and BLEND (Alg 4, Eq 11-14)            orc_weights/orc_blend
 *
 * Readings of passages that are silent, ambiguous or garbled (each one is
 * listed in the design notes):
 *  - PGS rows: contact = normal + two box-friction tangents bounded by
 *    +-mu*lambda_n (current lambda_n); ball joint = three world-axis rows with
 *    bounds +-inf.  Normal target -phi/h when phi > 0 (speculative), else
 *    erp*max(-phi - slop, 0)/h; joint target -erp*(e.(pB - pA))/h; no
 *    compliance (C = 0) -- Eq 2-4 written in the usual velocity-level form.
 *  - Gauss-Seidel order: constraints are coloured greedily per worker in
 *    descending priority mix64(kind<<62 ^ key) (SplitMix64 finaliser);
 *    sweeps go colour by colour, constraints in canonical order, rows
 *    normal, t1, t2 (joints x, y, z).  The paper does not colour (Bullet is
 *    sequential); constraints of one colour share no dynamic body, so the
 *    order inside a colour does not change any result.
 *  - Contact test: a pair is in contact when its gap phi <= margin.  Because
 *    that test decides an integer, it is evaluated in FP32 on FP32-rounded
 *    positions with the operation order written below.  Everything after
 *    the decision is FP64.  The tangent axis is the axis of the smallest
 *    |n_k|, a later axis winning only by more than ORC_TANGENT_TIE.
 *  - Alg 6 input = every current contact between two dynamic bodies in
 *    canonical (key) order; <W_x> = sum over workers in W_x of |P_w|, live;
 *    with the contact load (lb_load = 1; Section 6 proposes a load that
 *    follows contacts for scenes where bodies carry unequal contact counts)
 *    every active body counts 1 + the number of this step's contacts it is an
 *    end of (planes and static ends included), so <W_x> sums that weight over
 *    the active bodies of the workers in W_x;
 *    a load tie in the activation branch activates B in W_A; the gamma-ball
 *    activation uses W_A, W_B as read when the contact is taken up; the
 *    least-loaded choice of the equal-mask branch breaks ties towards the
 *    lowest worker index; the removal branches run only on steps whose index
 *    is a multiple of the removal cadence.  Alg 7 tests the body it is given
 *    (its "B" is that body b).
 *  - Alg 3 activates W_r \ W_b.  Alg 2 walks joints in index order over the
 *    joint graph.
 *  - Alg 5 / Eq 16: D(o,i) is the smallest BFS depth (1..beta) at which a body
 *    active only in worker i is met; unmet workers get weight 0 and a body
 *    with no worker met gets uniform weights.
 *  - Alg 4: the sign test compares q_i with q_0, the copy of the lowest-index
 *    worker; bodies outside O take their single copy unchanged.
 *  - Newly activated bodies start from the blended state (every worker reads
 *    the one blended state at the start of a step, Alg 1).
 *  - Learned warm start (not in the paper): 12 features per (worker,
 *    contact) pair, all taken from the blended state at the start of the
 *    step (before gravity) and made dimensionless with g_ref = max(|g|, 1):
 *      0-2  J v along n, t1, t2 (B minus A; static ends have v = 0) / (g_ref h)
 *      3    penetration max(-phi, 0) / (g_ref h^2)
 *      4-6  the previous-step impulses the plain warm start applies / s
 *      7-8  inverse masses of A and B (0 for a static end or a plane)
 *      9-10 degrees of A and B in G^t / 8 (0 for a static end)
 *      11   min over the dynamic ends of the BFS distance in G^t to the
 *           nearest body of O, capped at ORC_DEPTH_CAP, / ORC_DEPTH_CAP
 *    with s = k_n g_ref h, k_n = 1 / (im_A + im_B) over the dynamic ends:
 *    the impulse that cancels one step of gravity on the normal row.  Joint
 *    pairs have all-zero features and s = 0.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -std=c11 -shared -fPIC (no fused
 * multiply-add, so FP32 decisions round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_CAPACITY (-3)
#define ORC_ERR_MEMBERSHIP (-6)

#define ORC_MAX_COLOURS 256
#define ORC_DEPTH_CAP 8       /* depth feature: BFS levels searched from O */
#define ORC_NFEAT 12

typedef struct {
    double gravity[3];
    double margin;       /* contact when gap <= margin */
    double erp;          /* fraction of penetration / joint error removed per step */
    double slop;         /* penetration allowed before push-out */
    double warmstart;    /* factor on the previous step's impulses */
    int lb_activate;     /* Alg 6 activation branch enabled */
    int lb_deact_every;  /* Alg 6 removal branches on steps with index % k == 0; 0 = never */
    double res_tol;      /* > 0: a worker stops sweeping once its RMS residual <= res_tol */
    int res_check_every; /* sweeps between residual checks when res_tol > 0 */
    int lb_load;         /* 0: <W> counts active bodies (Table 1); 1: contact load (above) */
    int weights;         /* 0: Eq 15-16 weights; 1: uniform 1/|W_b| (the naive weights of Fig 8) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */

/* Threads for the loops whose iterations are independent (contacts per
 * body, PGS per worker, geodesic search per body); 1 (the default) runs
 * everything on the caller's thread.  No result depends on this number. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int orc_get_threads(void) { return g_threads; }

static int orc_thread_count(void) {
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

static int orc_thread_id(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz ? sz : 1);
    return p;
}

static int popc64(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

static int lowest_bit(uint64_t x) {
    for (int i = 0; i < 64; ++i) if (x >> i & 1u) return i;
    return -1;
}

/* SplitMix64 output function (Steele, Lea & Flood 2014), used as the
 * colouring priority. */
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void cross3(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* rotation matrix of a unit quaternion q = (w, x, y, z) */
static void quat_to_matrix(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void mat_vec(const double R[9], const double v[3], double out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = R[3 * i] * v[0] + R[3 * i + 1] * v[1] + R[3 * i + 2] * v[2];
}

/* Hamilton product a (x) b, quaternions as (w, x, y, z) */
static void quat_mul(const double a[4], const double b[4], double out[4]) {
    out[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    out[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    out[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    out[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* ------------------------------------------------------------------------ */
/* c1: contacts                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int a, b;        /* a < b; b >= n_bodies is plane (b - n_bodies) */
    double phi;      /* signed gap */
    double n[3];     /* unit normal from a towards b */
    double t1[3];    /* first tangent; t2 = n x t1 */
    int k;           /* point of a box manifold (0 for spheres) */
    int at_point;    /* box contact: both lever arms reach the point p */
    double p[3];
    double amb;      /* box contact: closeness of its decisions to their thresholds (bands) */
} orc_contact;

typedef struct { int64_t cx, cy, cz; int scene; int body; } cell_entry;

static int cmp_cell(const void *pa, const void *pb) {
    const cell_entry *a = pa, *b = pb;
    if (a->scene != b->scene) return a->scene < b->scene ? -1 : 1;
    if (a->cx != b->cx) return a->cx < b->cx ? -1 : 1;
    if (a->cy != b->cy) return a->cy < b->cy ? -1 : 1;
    if (a->cz != b->cz) return a->cz < b->cz ? -1 : 1;
    return a->body < b->body ? -1 : (a->body > b->body);
}

static int cmp_contact_key(const void *pa, const void *pb) {
    const orc_contact *a = pa, *b = pb;
    if (a->a != b->a) return a->a < b->a ? -1 : 1;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    return a->k < b->k ? -1 : (a->k > b->k);
}

/* FP32 contact decision for two spheres (integer outcome, evaluated in the
 * kernel's precision): d = cb - ca, |d|^2 <= (ra + rb + margin)^2. */
static int sphere_pair_touches_f32(const double *ca, const double *cb, double ra, double rb,
                                   double margin) {
    float ax = (float)ca[0], ay = (float)ca[1], az = (float)ca[2];
    float bx = (float)cb[0], by = (float)cb[1], bz = (float)cb[2];
    float dx = bx - ax, dy = by - ay, dz = bz - az;
    float dxx = dx * dx, dyy = dy * dy, dzz = dz * dz;
    float d2 = (dxx + dyy) + dzz;
    float rs = ((float)ra + (float)rb) + (float)margin;
    float rs2 = rs * rs;
    return d2 <= rs2;
}

/* FP32 plane decision: ((nx*px + ny*py) + nz*pz) - d - r <= margin. */
static int sphere_plane_touches_f32(const double *c, double r, const double *pl, double margin) {
    float px = (float)c[0], py = (float)c[1], pz = (float)c[2];
    float nx = (float)pl[0], ny = (float)pl[1], nz = (float)pl[2], d = (float)pl[3];
    float s0 = nx * px, s1 = ny * py, s2 = nz * pz;
    float dotp = (s0 + s1) + s2;
    float phi = (dotp - d) - (float)r;
    return phi <= (float)margin;
}

/* tangent axis: the smallest |n_k|, scanning x, y, z, a later axis winning
 * only when smaller by more than ORC_TANGENT_TIE (axis-aligned normals tie
 * exactly in two components; any precision accurate to well under the
 * tolerance picks the same axis) */
#define ORC_TANGENT_TIE 1e-4
static int tangent_axis(const double n[3]) {
    int k = 0;
    double m = fabs(n[0]);
    if (fabs(n[1]) < m - ORC_TANGENT_TIE) { k = 1; m = fabs(n[1]); }
    if (fabs(n[2]) < m - ORC_TANGENT_TIE) k = 2;
    return k;
}

static void tangent_from_axis(const double n[3], int k, double t1[3]) {
    double e[3] = {0, 0, 0};
    e[k] = 1.0;
    double ne = dot3(n, e);
    double t[3] = {e[0] - ne * n[0], e[1] - ne * n[1], e[2] - ne * n[2]};
    double L = sqrt(dot3(t, t));
    t1[0] = t[0] / L; t1[1] = t[1] / L; t1[2] = t[2] / L;
}

static void fill_sphere_contact(orc_contact *c, int a, int b, const double *ca, const double *cb,
                                double ra, double rb) {
    c->a = a; c->b = b; c->k = 0; c->at_point = 0; c->amb = INFINITY;
    double d[3] = {cb[0] - ca[0], cb[1] - ca[1], cb[2] - ca[2]};
    double L = sqrt(dot3(d, d));
    c->phi = L - ra - rb;
    if (L < 1e-12) {
        c->n[0] = 0; c->n[1] = 0; c->n[2] = 1;
    } else {
        c->n[0] = d[0] / L; c->n[1] = d[1] / L; c->n[2] = d[2] / L;
    }
    tangent_from_axis(c->n, tangent_axis(c->n), c->t1);
}

static void fill_plane_contact(orc_contact *c, int a, int b, const double *ca, double ra,
                               const double *pl) {
    c->a = a; c->b = b; c->k = 0; c->at_point = 0; c->amb = INFINITY;
    c->phi = dot3(pl, ca) - pl[3] - ra;
    /* normal from the sphere (a) towards the plane (b): minus the plane normal */
    c->n[0] = -pl[0]; c->n[1] = -pl[1]; c->n[2] = -pl[2];
    tangent_from_axis(c->n, tangent_axis(c->n), c->t1);
}

typedef struct {
    int n;
    const double *state;   /* n x 13 */
    const double *radius;
    const double *inv_mass;
    int n_planes;
    const double *planes;  /* np x 4 */
    const int *plane_scene;
    const int *scene_of_body;
    const int *scene_flags;
    double margin;
    const double *half;    /* n x 3 half extents (zeros: a sphere), or NULL: all spheres */
} contact_input;

/* FP64 box geometry (box_oracle.c); *amb: how close its decisions came to
 * their thresholds, in bands (< 1: an FP32 computation may decide otherwise) */
int box_plane(const double c[3], const double q[4], const double h[3], const double plane[4],
              double margin, double pts[12], double gaps[4], double normal[3], double *amb);
int sphere_box(const double s[3], double r, const double c[3], const double q[4], const double h[3],
               double margin, double pt[3], double normal[3], double *gap, double *amb);
int box_box(const double cA[3], const double qA[4], const double hA[3], const double cB[3],
            const double qB[4], const double hB[3], double margin, double pts[12], double gaps[4],
            double normal[3], int *axis, double *sep, double *amb);

static int is_box(const contact_input *in, int b) {
    return in->half && (in->half[3 * (size_t)b] > 0 || in->half[3 * (size_t)b + 1] > 0 ||
                        in->half[3 * (size_t)b + 2] > 0);
}

/* one point of a box contact (normal n from a towards b after the sign) */
static void fill_box_point(orc_contact *c, int a, int b, int k, const double p[3], double gap, const double n[3],
                           double sgn, double amb) {
    c->a = a; c->b = b; c->k = k; c->at_point = 1;
    c->phi = gap;
    c->amb = amb;
    for (int j = 0; j < 3; ++j) { c->p[j] = p[j]; c->n[j] = sgn * n[j]; }
    tangent_from_axis(c->n, tangent_axis(c->n), c->t1);
}

typedef struct { orc_contact *list; size_t cnt, cap; } contact_buf;

static orc_contact *cb_next(contact_buf *B) {
    if (B->cnt == B->cap) { B->cap *= 2; B->list = realloc(B->list, B->cap * sizeof(orc_contact)); }
    return &B->list[B->cnt++];
}

/* the contacts of a body pair with at least one box: the bounding spheres
 * must meet (the same FP32 test as for spheres), then the FP64 box
 * geometry decides; the normal runs from a towards b */
static void box_pair_contacts(const contact_input *in, int a, int b, contact_buf *B) {
    const double *ca = in->state + 13 * (size_t)a, *cb = in->state + 13 * (size_t)b;
    if (!sphere_pair_touches_f32(ca, cb, in->radius[a], in->radius[b], in->margin)) return;
    const double *ha = in->half + 3 * (size_t)a, *hb = in->half + 3 * (size_t)b;
    double pts[12], gaps[4], nrm[3], amb = INFINITY;
    if (is_box(in, a) && is_box(in, b)) {
        int axis;
        double sep;
        const int k = box_box(ca, ca + 3, ha, cb, cb + 3, hb, in->margin, pts, gaps, nrm, &axis, &sep, &amb);
        for (int i = 0; i < k; ++i) fill_box_point(cb_next(B), a, b, i, pts + 3 * i, gaps[i], nrm, 1.0, amb);
    } else {
        /* one sphere, one box: sphere_box's normal runs from the sphere to the box */
        const int sph = is_box(in, a) ? b : a, bx = sph == a ? b : a;
        const double *cs = in->state + 13 * (size_t)sph, *cx = in->state + 13 * (size_t)bx;
        double gap;
        if (sphere_box(cs, in->radius[sph], cx, cx + 3, in->half + 3 * (size_t)bx, in->margin, pts, nrm, &gap, &amb))
            fill_box_point(cb_next(B), a, b, 0, pts, gap, nrm, sph == a ? 1.0 : -1.0, amb);
    }
}

static void box_plane_contacts(const contact_input *in, int a, int p, contact_buf *B) {
    const double *ca = in->state + 13 * (size_t)a, *pl = in->planes + 4 * (size_t)p;
    if (!sphere_plane_touches_f32(ca, in->radius[a], pl, in->margin)) return;
    double pts[12], gaps[4], nrm[3], amb = INFINITY;
    const int k = box_plane(ca, ca + 3, in->half + 3 * (size_t)a, pl, in->margin, pts, gaps, nrm, &amb);
    for (int i = 0; i < k; ++i) fill_box_point(cb_next(B), a, in->n + p, i, pts + 3 * i, gaps[i], nrm, 1.0, amb);
}

/* All contacts of the current state in canonical order (ascending (a, b)).
 * Sphere pairs are found through a uniform grid whose cells are at least as
 * wide as the largest contact distance, so every touching pair lies in
 * neighbouring cells; the grid only prunes, every candidate is tested.
 * Pairs where both ends are static are skipped. Returns the count, or
 * ORC_ERR_CAPACITY if more than cap contacts exist (out is then partial). */
/* Sphere-sphere (or box) contacts (a, b > a) of body a through the sorted
 * cell list: for each of the 3 x 3 neighbouring (x, y) columns, one search
 * for the lowest cell z - 1, then a scan up to cell z + 1. */
static void grid_contacts_of(const contact_input *in, const cell_entry *cells, int n, double cs, int a,
                             contact_buf *B) {
    int s = in->scene_of_body[a];
    if (!(in->scene_flags[s] & 1)) return;
    const double *ca = in->state + 13 * (size_t)a;
    int64_t cx = (int64_t)floor(ca[0] / cs), cy = (int64_t)floor(ca[1] / cs), cz = (int64_t)floor(ca[2] / cs);
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
            cell_entry key = {cx + dx, cy + dy, cz - 1, s, -1};
            int lo = 0, hi = n;   /* lower bound of key */
            while (lo < hi) {
                int mid = (lo + hi) / 2;
                if (cmp_cell(&cells[mid], &key) < 0) lo = mid + 1; else hi = mid;
            }
            for (int k = lo; k < n; ++k) {
                const cell_entry *e = &cells[k];
                if (e->scene != s || e->cx != key.cx || e->cy != key.cy || e->cz > cz + 1) break;
                int b = e->body;
                if (b <= a) continue;
                if (in->inv_mass[a] == 0 && in->inv_mass[b] == 0) continue;
                const double *cb = in->state + 13 * (size_t)b;
                if (is_box(in, a) || is_box(in, b))
                    box_pair_contacts(in, a, b, B);
                else if (sphere_pair_touches_f32(ca, cb, in->radius[a], in->radius[b], in->margin))
                    fill_sphere_contact(cb_next(B), a, b, ca, cb, in->radius[a], in->radius[b]);
            }
        }
}

static int64_t contacts_impl(const contact_input *in, int use_grid, orc_contact **out_list) {
    int n = in->n;
    size_t cap = 1024, cnt = 0;
    orc_contact *list = malloc(cap * sizeof(orc_contact));
#define PUSH_CONTACT(expr)                                                         \
    do {                                                                           \
        if (cnt == cap) { cap *= 2; list = realloc(list, cap * sizeof(orc_contact)); } \
        expr;                                                                      \
        ++cnt;                                                                     \
    } while (0)
    double rmax = 0;
    for (int i = 0; i < n; ++i) if (in->radius[i] > rmax) rmax = in->radius[i];
    if (use_grid && n > 0) {
        double cs = (2.0 * rmax + in->margin) * 1.01;
        cell_entry *cells = malloc((size_t)n * sizeof(cell_entry));
        for (int i = 0; i < n; ++i) {
            const double *c = in->state + 13 * (size_t)i;
            cells[i].cx = (int64_t)floor(c[0] / cs);
            cells[i].cy = (int64_t)floor(c[1] / cs);
            cells[i].cz = (int64_t)floor(c[2] / cs);
            cells[i].scene = in->scene_of_body[i];
            cells[i].body = i;
        }
        qsort(cells, n, sizeof(cell_entry), cmp_cell);
        /* bodies are independent here: each thread collects its own list and
         * the lists are joined before the canonical sort below */
        int nt = orc_thread_count();
        contact_buf *part = calloc((size_t)nt, sizeof(contact_buf));
        for (int t = 0; t < nt; ++t) { part[t].cap = 1024; part[t].list = malloc(1024 * sizeof(orc_contact)); }
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
        for (int a = 0; a < n; ++a) grid_contacts_of(in, cells, n, cs, a, &part[orc_thread_id()]);
        for (int t = 0; t < nt; ++t) {
            for (size_t i = 0; i < part[t].cnt; ++i) PUSH_CONTACT(list[cnt] = part[t].list[i]);
            free(part[t].list);
        }
        free(part);
        free(cells);
    } else {
        for (int a = 0; a < n; ++a) {
            int s = in->scene_of_body[a];
            if (!(in->scene_flags[s] & 1)) continue;
            const double *ca = in->state + 13 * (size_t)a;
            for (int b = a + 1; b < n; ++b) {
                if (in->scene_of_body[b] != s) continue;
                if (in->inv_mass[a] == 0 && in->inv_mass[b] == 0) continue;
                const double *cb = in->state + 13 * (size_t)b;
                if (is_box(in, a) || is_box(in, b)) {
                    contact_buf B = {list, cnt, cap};
                    box_pair_contacts(in, a, b, &B);
                    list = B.list; cnt = B.cnt; cap = B.cap;
                } else if (sphere_pair_touches_f32(ca, cb, in->radius[a], in->radius[b], in->margin))
                    PUSH_CONTACT(fill_sphere_contact(&list[cnt], a, b, ca, cb, in->radius[a], in->radius[b]));
            }
        }
    }
    for (int a = 0; a < n; ++a) {
        if (in->inv_mass[a] == 0) continue;
        const double *ca = in->state + 13 * (size_t)a;
        for (int p = 0; p < in->n_planes; ++p) {
            if (in->plane_scene[p] != in->scene_of_body[a]) continue;
            const double *pl = in->planes + 4 * (size_t)p;
            if (is_box(in, a)) {
                contact_buf B = {list, cnt, cap};
                box_plane_contacts(in, a, p, &B);
                list = B.list; cnt = B.cnt; cap = B.cap;
            } else if (sphere_plane_touches_f32(ca, in->radius[a], pl, in->margin))
                PUSH_CONTACT(fill_plane_contact(&list[cnt], a, n + p, ca, in->radius[a], pl));
        }
    }
#undef PUSH_CONTACT
    qsort(list, cnt, sizeof(orc_contact), cmp_contact_key);
    *out_list = list;
    return (int64_t)cnt;
}

/* Standalone entry point: contacts of a state; writes up to cap contacts.
 * Returns the total number found (may exceed cap). */
int64_t orc_contacts(int n, const double *state, const double *radius, const double *inv_mass,
                     int n_planes, const double *planes, const int *plane_scene,
                     const int *scene_of_body, const int *scene_flags, double margin, int use_grid,
                     int64_t cap, int *out_ab, double *out_phi, double *out_n, double *out_t1) {
    contact_input in = {n, state, radius, inv_mass, n_planes, planes, plane_scene, scene_of_body,
                        scene_flags, margin, NULL};
    orc_contact *list = NULL;
    int64_t cnt = contacts_impl(&in, use_grid, &list);
    for (int64_t i = 0; i < cnt && i < cap; ++i) {
        out_ab[2 * i] = list[i].a; out_ab[2 * i + 1] = list[i].b;
        out_phi[i] = list[i].phi;
        for (int k = 0; k < 3; ++k) { out_n[3 * i + k] = list[i].n[k]; out_t1[3 * i + k] = list[i].t1[k]; }
    }
    free(list);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* c2: constraint graph G^t (Section 5.1): vertices are bodies, an undirected  */
/* edge joins two dynamic bodies linked by a contact or a joint; static       */
/* bodies carry no edges; adjacency lists sorted ascending, duplicates merged. */
/* ------------------------------------------------------------------------ */

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return x < y ? -1 : (x > y);
}

/* edges given as pairs (u[i], v[i]); entries with a negative end or a static
 * end are ignored.  row_ptr has n+1 entries; returns the adjacency length. */
static int64_t build_graph(int n, const double *inv_mass, int64_t ne, const int *eu, const int *ev,
                           int **out_row_ptr, int **out_col) {
    int *deg = xcalloc((size_t)n + 1, sizeof(int));
    for (int64_t i = 0; i < ne; ++i) {
        int u = eu[i], v = ev[i];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) continue;
        if (inv_mass[u] == 0 || inv_mass[v] == 0) continue;
        deg[u]++; deg[v]++;
    }
    int *tmp_ptr = xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i) tmp_ptr[i + 1] = tmp_ptr[i] + deg[i];
    int *tmp = xcalloc((size_t)tmp_ptr[n] + 1, sizeof(int));
    int *fill = xcalloc((size_t)n + 1, sizeof(int));
    for (int64_t i = 0; i < ne; ++i) {
        int u = eu[i], v = ev[i];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) continue;
        if (inv_mass[u] == 0 || inv_mass[v] == 0) continue;
        tmp[tmp_ptr[u] + fill[u]++] = v;
        tmp[tmp_ptr[v] + fill[v]++] = u;
    }
    int *row_ptr = xcalloc((size_t)n + 1, sizeof(int));
    int *col = xcalloc((size_t)tmp_ptr[n] + 1, sizeof(int));
    int64_t m = 0;
    for (int i = 0; i < n; ++i) {
        int *seg = tmp + tmp_ptr[i];
        int len = tmp_ptr[i + 1] - tmp_ptr[i];
        qsort(seg, len, sizeof(int), cmp_int);
        row_ptr[i] = (int)m;
        for (int k = 0; k < len; ++k)
            if (k == 0 || seg[k] != seg[k - 1]) col[m++] = seg[k];
    }
    row_ptr[n] = (int)m;
    free(deg); free(tmp_ptr); free(tmp); free(fill);
    *out_row_ptr = row_ptr;
    *out_col = col;
    return m;
}

int64_t orc_graph(int n, const double *inv_mass, int64_t ne, const int *eu, const int *ev,
                  int64_t cap, int *row_ptr_out, int *col_out) {
    int *rp, *col;
    int64_t m = build_graph(n, inv_mass, ne, eu, ev, &rp, &col);
    memcpy(row_ptr_out, rp, ((size_t)n + 1) * sizeof(int));
    for (int64_t i = 0; i < m && i < cap; ++i) col_out[i] = col[i];
    free(rp); free(col);
    return m;
}

/* ------------------------------------------------------------------------ */
/* BFS helper: getBFSVertices(root, depth) = every vertex at graph distance   */
/* 0..depth from root, root included (the gamma-balls of Alg 3 and Alg 6).    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    int *stamp;
    int *dist;
    int *queue;
    int cur;
} bfs_ws;

static void bfs_ws_init(bfs_ws *w, int n) {
    w->n = n;
    w->stamp = xcalloc((size_t)n + 1, sizeof(int));
    w->dist = xcalloc((size_t)n + 1, sizeof(int));
    w->queue = xcalloc((size_t)n + 1, sizeof(int));
    w->cur = 0;
}

static void bfs_ws_free(bfs_ws *w) { free(w->stamp); free(w->dist); free(w->queue); }

/* fills w->queue[0..count) with the vertices in BFS order; returns count */
static int bfs_vertices(bfs_ws *w, const int *row_ptr, const int *col, int root, int depth) {
    w->cur++;
    int head = 0, tail = 0;
    w->queue[tail++] = root;
    w->stamp[root] = w->cur;
    w->dist[root] = 0;
    while (head < tail) {
        int u = w->queue[head++];
        if (w->dist[u] >= depth) continue;
        for (int k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            int v = col[k];
            if (w->stamp[v] == w->cur) continue;
            w->stamp[v] = w->cur;
            w->dist[v] = w->dist[u] + 1;
            w->queue[tail++] = v;
        }
    }
    return tail;
}

/* ------------------------------------------------------------------------ */
/* Membership edits (Table 1: activate / deactivate), with live |P_w| counts  */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t *mask;        /* per body, bit w = scene-local worker w */
    const int *sob;        /* scene of body */
    const int *part_base;  /* global index of worker 0 of each scene */
    int64_t *count;        /* load per global worker: sum of the weights of its active bodies */
    const int64_t *weight; /* per body; NULL: every body weighs 1, the count |P_w| */
} membership;

static int64_t body_weight(const membership *m, int b) { return m->weight ? m->weight[b] : 1; }

static void activate(membership *m, uint64_t W, int b) {
    uint64_t add = W & ~m->mask[b];
    int base = m->part_base[m->sob[b]];
    for (int w = 0; w < 64; ++w) if (add >> w & 1u) m->count[base + w] += body_weight(m, b);
    m->mask[b] |= add;
}

static void deactivate(membership *m, uint64_t W, int b) {
    uint64_t rem = W & m->mask[b];
    int base = m->part_base[m->sob[b]];
    for (int w = 0; w < 64; ++w) if (rem >> w & 1u) m->count[base + w] -= body_weight(m, b);
    m->mask[b] &= ~rem;
}

/* <W_x>: total number of active bodies over the workers in W_x (Table 1),
 * each body counted with its weight */
static int64_t load_of(const membership *m, uint64_t W, int scene) {
    int64_t s = 0;
    int base = m->part_base[scene];
    for (int w = 0; w < 64; ++w) if (W >> w & 1u) s += m->count[base + w];
    return s;
}

/* Alg 7: b is a bridge body when the union of its neighbours' workers has
 * more than one worker. */
static int is_bridge(const membership *m, const int *row_ptr, const int *col, int b) {
    uint64_t W = 0;
    for (int k = row_ptr[b]; k < row_ptr[b + 1]; ++k) W |= m->mask[col[k]];
    return popc64(W) > 1;
}

/* Alg 6 over the given contacts (pairs of dynamic bodies, canonical order). */
static void load_balance_impl(membership *m, int n, const int *row_ptr, const int *col,
                              int64_t nc, const int *ca, const int *cb, const int *scene_gamma,
                              int do_activate, int do_deactivate) {
    bfs_ws ws;
    bfs_ws_init(&ws, n);
    for (int64_t c = 0; c < nc; ++c) {
        int A = ca[c], B = cb[c];
        uint64_t WA = m->mask[A], WB = m->mask[B];          /* masks as read now */
        int scene = m->sob[A];
        if ((WA & WB) == 0) {                                /* activation branch */
            if (!do_activate) continue;
            int root;
            if (load_of(m, WA, scene) <= load_of(m, WB, scene)) {  /* ties: B joins W_A */
                activate(m, WA, B);
                root = B;
            } else {
                activate(m, WB, A);
                root = A;
            }
            int cnt = bfs_vertices(&ws, row_ptr, col, root, scene_gamma[scene]);  /* gamma-ball */
            for (int k = 0; k < cnt; ++k) {
                int v = ws.queue[k];
                activate(m, (WA | WB) & ~m->mask[v], v);
            }
        } else if (!do_deactivate) {
            continue;
        } else if (popc64(WA) > 1 && popc64(WB) == 1 && !is_bridge(m, row_ptr, col, A)) {
            deactivate(m, WA & ~WB, A);
        } else if (popc64(WB) > 1 && popc64(WA) == 1 && !is_bridge(m, row_ptr, col, B)) {
            deactivate(m, WB & ~WA, B);
        } else if (WA == WB) {                               /* equal masks */
            int base = m->part_base[scene];
            int s = -1;
            int64_t best = 0;
            for (int w = 0; w < 64; ++w) {                   /* least loaded, ties -> lowest */
                if (!(WA >> w & 1u)) continue;
                if (s < 0 || m->count[base + w] < best) { s = w; best = m->count[base + w]; }
            }
            uint64_t keep = (uint64_t)1 << s;
            deactivate(m, WA & ~keep, A);
            deactivate(m, WB & ~keep, B);
        }
    }
    bfs_ws_free(&ws);
}

static int64_t *counts_from_masks(int n, const uint64_t *mask, const int *sob, const int *part_base,
                                  int n_parts_total, const int64_t *weight) {
    int64_t *count = xcalloc((size_t)n_parts_total + 1, sizeof(int64_t));
    for (int b = 0; b < n; ++b)
        for (int w = 0; w < 64; ++w)
            if (mask[b] >> w & 1u) count[part_base[sob[b]] + w] += weight ? weight[b] : 1;
    return count;
}

/* Standalone Alg 6: masks updated in place; weight NULL = body counts. */
void orc_load_balance(int n, uint64_t *mask, const int *scene_of_body, const int *part_base,
                      int n_parts_total, const int *row_ptr, const int *col, int64_t nc,
                      const int *ca, const int *cb, const int *scene_gamma, int do_activate,
                      int do_deactivate, const int64_t *weight) {
    int64_t *count = counts_from_masks(n, mask, scene_of_body, part_base, n_parts_total, weight);
    membership m = {mask, scene_of_body, part_base, count, weight};
    load_balance_impl(&m, n, row_ptr, col, nc, ca, cb, scene_gamma, do_activate, do_deactivate);
    free(count);
}

int orc_is_bridge(int n, const uint64_t *mask, const int *row_ptr, const int *col, int b) {
    (void)n;
    membership m = {(uint64_t *)mask, NULL, NULL, NULL, NULL};
    return is_bridge(&m, row_ptr, col, b);
}

/* ------------------------------------------------------------------------ */
/* Alg 2 + Alg 3: overlap assignment for articulated bodies over joints.      */
/* ------------------------------------------------------------------------ */

static void grow_overlap(membership *m, bfs_ws *ws, const int *row_ptr, const int *col, int root,
                         int gamma, uint64_t Wr) {
    int cnt = bfs_vertices(ws, row_ptr, col, root, gamma);   /* Alg 3 gamma-ball */
    for (int k = 0; k < cnt; ++k) {
        int b = ws->queue[k];
        if (popc64(m->mask[b]) >= 2) continue;                /* b already in O */
        activate(m, Wr & ~m->mask[b], b);                     /* W_r \ W_b */
    }
}

/* masks updated in place; joints with a world end or a static end are skipped
 * (they are not edges of G).  The BFS runs on the joint graph. */
void orc_assign_overlap(int n, uint64_t *mask, const int *scene_of_body, const int *part_base,
                        int n_parts_total, const double *inv_mass, int nj, const int *joint_ab,
                        const int *scene_gamma) {
    int *eu = xcalloc((size_t)nj + 1, sizeof(int)), *ev = xcalloc((size_t)nj + 1, sizeof(int));
    for (int j = 0; j < nj; ++j) { eu[j] = joint_ab[2 * j]; ev[j] = joint_ab[2 * j + 1]; }
    int *row_ptr, *col;
    build_graph(n, inv_mass, nj, eu, ev, &row_ptr, &col);
    int64_t *count = counts_from_masks(n, mask, scene_of_body, part_base, n_parts_total, NULL);
    membership m = {mask, scene_of_body, part_base, count, NULL};
    bfs_ws ws;
    bfs_ws_init(&ws, n);
    for (int j = 0; j < nj; ++j) {                              /* Alg 2: joints in order */
        int A = eu[j], B = ev[j];
        if (A < 0 || B < 0 || inv_mass[A] == 0 || inv_mass[B] == 0 || A == B) continue;
        uint64_t WA = mask[A], WB = mask[B];
        if (popc64(WA) == 1 && popc64(WB) == 1 && WA != WB) {   /* joint across workers */
            int gamma = scene_gamma[scene_of_body[A]];
            activate(&m, mask[B], A);
            grow_overlap(&m, &ws, row_ptr, col, A, gamma, mask[A] | mask[B]);
            activate(&m, mask[A], B);
            grow_overlap(&m, &ws, row_ptr, col, B, gamma, mask[A] | mask[B]);
        }
    }
    bfs_ws_free(&ws);
    free(count); free(row_ptr); free(col); free(eu); free(ev);
}

/* ------------------------------------------------------------------------ */
/* c7: D(o,i) (Eq 16), searched breadth-first up to beta as in Alg 5.         */
/* Entries are ordered by body, then worker; D has one byte per entry, 255   */
/* where the worker is not met within beta (and for bodies outside O).        */
/* ------------------------------------------------------------------------ */

/* D(o, i) of one body o (its entries of D); ws is the caller's workspace */
static void geodesics_of(bfs_ws *ws, int o, const uint64_t *mask, const int *sob, const int *scene_beta,
                         const int *row_ptr, const int *col, const int64_t *entry_ptr, uint8_t *D) {
    uint64_t Wo = mask[o];
    for (int64_t e = entry_ptr[o]; e < entry_ptr[o + 1]; ++e) D[e] = 255;
    if (popc64(Wo) < 2) return;
    int beta = scene_beta[sob[o]];
    /* breadth-first from o, depth 1..beta (Alg 5); the first body met
     * that is active only in worker i, with i in W_o, gives the minimum
     * of Eq 16 for i */
    ws->cur++;
    int head = 0, tail = 0;
    ws->queue[tail++] = o;
    ws->stamp[o] = ws->cur;
    ws->dist[o] = 0;
    uint64_t found = 0;
    while (head < tail && found != Wo) {
        int u = ws->queue[head++];
        if (ws->dist[u] >= beta) continue;
        for (int k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            int v = col[k];
            if (ws->stamp[v] == ws->cur) continue;
            ws->stamp[v] = ws->cur;
            ws->dist[v] = ws->dist[u] + 1;
            ws->queue[tail++] = v;
            uint64_t Wv = mask[v];
            if (popc64(Wv) == 1 && (Wv & Wo) == Wv && !(found & Wv)) {
                found |= Wv;
                int w = lowest_bit(Wv);
                int rank = popc64(Wo & (((uint64_t)1 << w) - 1));
                D[entry_ptr[o] + rank] = (uint8_t)ws->dist[v];
            }
        }
    }
    /* stopping once every worker is met (as Alg 5 does) changes nothing:
     * later hits are at the same or a larger depth and are not recorded */
}

/* every body's search is its own (it writes only its entries of D), so the
 * bodies may be taken by several threads, each with its own workspace */
static void geodesics_impl(int n, const uint64_t *mask, const int *sob, const int *scene_beta,
                           const int *row_ptr, const int *col, const int64_t *entry_ptr,
                           uint8_t *D) {
#pragma omp parallel num_threads(orc_thread_count())
    {
        bfs_ws ws;
        bfs_ws_init(&ws, n);
#pragma omp for schedule(dynamic, 64)
        for (int o = 0; o < n; ++o) geodesics_of(&ws, o, mask, sob, scene_beta, row_ptr, col, entry_ptr, D);
        bfs_ws_free(&ws);
    }
}

void orc_geodesics(int n, const uint64_t *mask, const int *scene_of_body, const int *scene_beta,
                   const int *row_ptr, const int *col, uint8_t *D_out) {
    int64_t *entry_ptr = xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int b = 0; b < n; ++b) entry_ptr[b + 1] = entry_ptr[b] + popc64(mask[b]);
    geodesics_impl(n, mask, scene_of_body, scene_beta, row_ptr, col, entry_ptr, D_out);
    free(entry_ptr);
}

/* c8: convex weights of Eq 15 from inverse distances; unmet workers weigh 0
 * and a body that met none gets uniform weights. */
void orc_weights(int k, const uint8_t *D, double *w) {
    double s = 0;
    for (int i = 0; i < k; ++i) {
        w[i] = (D[i] != 255) ? 1.0 / (double)D[i] : 0.0;
        s += w[i];
    }
    for (int i = 0; i < k; ++i) w[i] = (s > 0) ? w[i] / s : 1.0 / (double)k;
}

/* c9: Alg 4 over k copies (13 values each, workers in ascending order). */
void orc_blend(int k, const double *copies, const double *w, double *out) {
    double x[3] = {0, 0, 0}, v[3] = {0, 0, 0}, om[3] = {0, 0, 0}, q[4] = {0, 0, 0, 0};
    const double *q0 = copies + 3;
    for (int i = 0; i < k; ++i) {
        const double *s = copies + 13 * (size_t)i;
        for (int a = 0; a < 3; ++a) {
            x[a] += w[i] * s[a];          /* Eq 11 */
            v[a] += w[i] * s[7 + a];      /* Eq 12 */
            om[a] += w[i] * s[10 + a];    /* Eq 13 */
        }
        double qi[4] = {s[3], s[4], s[5], s[6]};
        double dq = qi[0] * q0[0] + qi[1] * q0[1] + qi[2] * q0[2] + qi[3] * q0[3];
        if (i > 0 && dq < 0) for (int a = 0; a < 4; ++a) qi[a] = -qi[a];   /* Alg 4 sign test */
        for (int a = 0; a < 4; ++a) q[a] += w[i] * qi[a];                  /* Eq 14 */
    }
    double L = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);  /* Alg 4 normalisation */
    for (int a = 0; a < 3; ++a) { out[a] = x[a]; out[7 + a] = v[a]; out[10 + a] = om[a]; }
    for (int a = 0; a < 4; ++a) out[3 + a] = q[a] / L;
}

/* ------------------------------------------------------------------------ */
/* c5: greedy first-fit colouring in descending priority.                    */
/* nodes: for each node its two dynamic body ids (-1 = none) and priority.   */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t prio; int idx; } prio_item;

static int cmp_prio_desc(const void *pa, const void *pb) {
    const prio_item *a = pa, *b = pb;
    if (a->prio != b->prio) return a->prio > b->prio ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* body_slots: 2 per node, local body indices in [0, n_local) or -1.
 * colour_out: one per node.  Returns the number of colours, or
 * ORC_ERR_CAPACITY beyond ORC_MAX_COLOURS. */
static int colour_nodes(int n_nodes, const int *body_slots, const uint64_t *prio, int n_local,
                        int *colour_out) {
    const int W = ORC_MAX_COLOURS / 64;
    uint64_t *used = xcalloc((size_t)n_local * W + 1, sizeof(uint64_t));
    prio_item *order = xcalloc((size_t)n_nodes + 1, sizeof(prio_item));
    for (int i = 0; i < n_nodes; ++i) { order[i].prio = prio[i]; order[i].idx = i; }
    qsort(order, n_nodes, sizeof(prio_item), cmp_prio_desc);
    int ncol = 0, err = 0;
    for (int r = 0; r < n_nodes; ++r) {
        int u = order[r].idx;
        int sa = body_slots[2 * u], sb = body_slots[2 * u + 1];
        int c = -1;
        for (int cc = 0; cc < ORC_MAX_COLOURS; ++cc) {
            int wd = cc / 64, bit = cc % 64;
            int taken = 0;
            if (sa >= 0 && (used[(size_t)sa * W + wd] >> bit & 1u)) taken = 1;
            if (sb >= 0 && (used[(size_t)sb * W + wd] >> bit & 1u)) taken = 1;
            if (!taken) { c = cc; break; }
        }
        if (c < 0) { err = 1; c = 0; }
        colour_out[u] = c;
        if (sa >= 0) used[(size_t)sa * W + c / 64] |= (uint64_t)1 << (c % 64);
        if (sb >= 0) used[(size_t)sb * W + c / 64] |= (uint64_t)1 << (c % 64);
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used); free(order);
    return err ? ORC_ERR_CAPACITY : ncol;
}

int orc_colour(int n_nodes, const int *body_slots, const uint64_t *prio, int n_local,
               int *colour_out) {
    return colour_nodes(n_nodes, body_slots, prio, n_local, colour_out);
}

/* ------------------------------------------------------------------------ */
/* The simulation: state, membership, warm-start cache, last-step records.   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int part;           /* global worker */
    uint64_t key;       /* kind<<62 | key */
    double lam[3];
} ws_item;

static int cmp_ws(const void *pa, const void *pb) {
    const ws_item *a = pa, *b = pb;
    if (a->part != b->part) return a->part < b->part ? -1 : 1;
    return a->key < b->key ? -1 : (a->key > b->key);
}

typedef struct {
    orc_params P;
    int n, np, nj, ns;
    double *st;          /* n x 13 blended state */
    double *rad, *im, *iI;
    double *planes; int *plane_scene;
    int *jab; double *janc;
    int *sob; double *mu, *dt; int *sflags, *sgamma, *sbeta, *nsets, *part_base;
    int n_parts;
    uint64_t *mask;
    ws_item *ws; int64_t ws_n;
    int64_t step_index;
    /* last step */
    orc_contact *con; int64_t nc;
    int *row_ptr, *col; int64_t nadj;
    int64_t *entry_ptr; int64_t ne;
    int *entry_part;
    uint8_t *D;
    double *weight;
    double *copies;     /* ne x 13 */
    /* pairs: (worker, constraint) in worker order, canonical inside */
    int64_t npairs;
    int *pair_part; int *pair_kind; int64_t *pair_cidx; uint64_t *pair_key; int *pair_colour;
    double *pair_lam;   /* npairs x 3 */
    double *pair_feat;  /* npairs x ORC_NFEAT learned-warm-start features */
    double *pair_scale; /* npairs: s = k_n g_ref h (0 for joints) */
    int *pair_found;    /* npairs: 1 if the previous step left impulses for it */
    uint8_t *depth;     /* n: BFS distance in G^t to O, capped at ORC_DEPTH_CAP */
    int *part_iters; double *part_res_sq, *part_res_max; int64_t *part_rows; int *part_colours;
    double res_sq_total; double res_max; int64_t res_rows;
    double joint_violation_max, joint_violation_sum;
    double *half;       /* n x 3 half extents (zeros: a sphere); NULL until orc_set_shapes */
} orc_sim;

/* Position-level joint violation of the current state (Section 6's error
 * measure for jointed scenes): per ball joint the gap |p_B - p_A| between its
 * pivots, p = x + R(q) anchor for a body end, the anchor for a world end.
 * out[0] = sum over joints, out[1] = largest gap. */
void orc_joint_error(const orc_sim *s, double *out);

orc_sim *orc_create(const orc_params *P, int n, const double *state13, const double *radius,
                    const double *inv_mass, int n_planes, const double *planes,
                    const int *plane_scene, int n_joints, const int *joint_ab,
                    const double *joint_anchors, int n_scenes, const int *scene_of_body,
                    const double *scene_mu, const double *scene_dt, const int *scene_flags,
                    const int *scene_gamma, const int *scene_beta, const int *n_sets) {
    orc_sim *s = xcalloc(1, sizeof(orc_sim));
    s->P = *P;
    s->n = n; s->np = n_planes; s->nj = n_joints; s->ns = n_scenes;
    s->st = xcalloc((size_t)n * 13 + 1, sizeof(double));
    memcpy(s->st, state13, (size_t)n * 13 * sizeof(double));
    s->rad = xcalloc((size_t)n + 1, sizeof(double));
    s->im = xcalloc((size_t)n + 1, sizeof(double));
    s->iI = xcalloc((size_t)n + 1, sizeof(double));
    for (int i = 0; i < n; ++i) {
        s->rad[i] = radius[i];
        s->im[i] = inv_mass[i];
        /* solid sphere: I = (2/5) m r^2, isotropic */
        s->iI[i] = inv_mass[i] > 0 ? inv_mass[i] / (0.4 * radius[i] * radius[i]) : 0.0;
    }
    s->planes = xcalloc((size_t)n_planes * 4 + 1, sizeof(double));
    memcpy(s->planes, planes, (size_t)n_planes * 4 * sizeof(double));
    s->plane_scene = xcalloc((size_t)n_planes + 1, sizeof(int));
    memcpy(s->plane_scene, plane_scene, (size_t)n_planes * sizeof(int));
    s->jab = xcalloc((size_t)n_joints * 2 + 1, sizeof(int));
    memcpy(s->jab, joint_ab, (size_t)n_joints * 2 * sizeof(int));
    s->janc = xcalloc((size_t)n_joints * 6 + 1, sizeof(double));
    memcpy(s->janc, joint_anchors, (size_t)n_joints * 6 * sizeof(double));
    s->sob = xcalloc((size_t)n + 1, sizeof(int));
    memcpy(s->sob, scene_of_body, (size_t)n * sizeof(int));
    s->mu = xcalloc((size_t)n_scenes, sizeof(double));
    s->dt = xcalloc((size_t)n_scenes, sizeof(double));
    s->sflags = xcalloc((size_t)n_scenes, sizeof(int));
    s->sgamma = xcalloc((size_t)n_scenes, sizeof(int));
    s->sbeta = xcalloc((size_t)n_scenes, sizeof(int));
    s->nsets = xcalloc((size_t)n_scenes, sizeof(int));
    s->part_base = xcalloc((size_t)n_scenes + 1, sizeof(int));
    for (int i = 0; i < n_scenes; ++i) {
        s->mu[i] = scene_mu[i]; s->dt[i] = scene_dt[i]; s->sflags[i] = scene_flags[i];
        s->sgamma[i] = scene_gamma[i]; s->sbeta[i] = scene_beta[i]; s->nsets[i] = n_sets[i];
        s->part_base[i + 1] = s->part_base[i] + n_sets[i];
    }
    s->n_parts = s->part_base[n_scenes];
    s->mask = xcalloc((size_t)n + 1, sizeof(uint64_t));
    return s;
}

/* Box bodies (row f1): half extents per body, zeros for a sphere.  Inverse
 * masses stay as given; a box's world inverse inertia R diag(1/I) R^T, I_k =
 * m/3 (h_j^2 + h_l^2), is formed from its orientation at every step.
 * Returns 0, or -1 for a negative extent. */
int orc_set_shapes(orc_sim *s, const double *half) {
    for (int i = 0; i < 3 * s->n; ++i)
        if (half[i] < 0) return -1;
    free(s->half);
    s->half = xcalloc((size_t)s->n * 3 + 1, sizeof(double));
    memcpy(s->half, half, (size_t)s->n * 3 * sizeof(double));
    return 0;
}

static int body_is_box(const orc_sim *s, int b) {
    return s->half && (s->half[3 * (size_t)b] > 0 || s->half[3 * (size_t)b + 1] > 0 || s->half[3 * (size_t)b + 2] > 0);
}

static void free_step_records(orc_sim *s) {
    free(s->con); s->con = NULL;
    free(s->row_ptr); free(s->col); s->row_ptr = s->col = NULL;
    free(s->entry_ptr); free(s->entry_part); s->entry_ptr = NULL; s->entry_part = NULL;
    free(s->D); free(s->weight); free(s->copies); s->D = NULL; s->weight = NULL; s->copies = NULL;
    free(s->pair_part); free(s->pair_kind); free(s->pair_cidx); free(s->pair_key);
    free(s->pair_colour); free(s->pair_lam);
    s->pair_part = s->pair_kind = s->pair_colour = NULL; s->pair_cidx = NULL; s->pair_key = NULL;
    s->pair_lam = NULL;
    free(s->pair_feat); free(s->pair_scale); free(s->pair_found); free(s->depth);
    s->pair_feat = NULL; s->pair_scale = NULL; s->pair_found = NULL; s->depth = NULL;
    free(s->part_iters); free(s->part_res_sq); free(s->part_res_max); free(s->part_rows); free(s->part_colours);
    s->part_iters = NULL; s->part_res_sq = NULL; s->part_res_max = NULL; s->part_rows = NULL; s->part_colours = NULL;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free_step_records(s);
    free(s->st); free(s->rad); free(s->im); free(s->iI); free(s->planes); free(s->plane_scene);
    free(s->jab); free(s->janc); free(s->sob); free(s->mu); free(s->dt); free(s->sflags);
    free(s->sgamma); free(s->sbeta); free(s->nsets); free(s->part_base); free(s->mask); free(s->ws);
    free(s->half);
    free(s);
}

/* initial partition: each body's single worker (scene-local index) */
int orc_set_partition(orc_sim *s, const int *set_of_body) {
    for (int b = 0; b < s->n; ++b) {
        if (s->im[b] == 0) { s->mask[b] = 0; continue; }
        int w = set_of_body[b];
        if (w < 0 || w >= s->nsets[s->sob[b]] || w >= 64) return ORC_ERR_MEMBERSHIP;
        s->mask[b] = (uint64_t)1 << w;
    }
    return ORC_OK;
}

int orc_set_masks(orc_sim *s, const uint64_t *mask) {
    for (int b = 0; b < s->n; ++b) {
        if (s->im[b] == 0) { s->mask[b] = 0; continue; }
        int ns = s->nsets[s->sob[b]];
        uint64_t allowed = ns >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << ns) - 1);
        if (mask[b] == 0 || (mask[b] & ~allowed)) return ORC_ERR_MEMBERSHIP;
        s->mask[b] = mask[b];
    }
    return ORC_OK;
}

void orc_get_masks(const orc_sim *s, uint64_t *out) { memcpy(out, s->mask, (size_t)s->n * sizeof(uint64_t)); }
void orc_set_state(orc_sim *s, const double *st) { memcpy(s->st, st, (size_t)s->n * 13 * sizeof(double)); }
void orc_get_state(const orc_sim *s, double *st) { memcpy(st, s->st, (size_t)s->n * 13 * sizeof(double)); }
void orc_set_step_index(orc_sim *s, int64_t k) { s->step_index = k; }
int64_t orc_get_step_index(const orc_sim *s) { return s->step_index; }

int orc_assign(orc_sim *s) {
    orc_assign_overlap(s->n, s->mask, s->sob, s->part_base, s->n_parts, s->im, s->nj, s->jab,
                       s->sgamma);
    return ORC_OK;
}

/* warm-start cache: n items (global worker, kind<<62|key, lambda[3]) */
void orc_set_warmstart(orc_sim *s, int64_t n, const int *part, const uint64_t *key,
                       const double *lam) {
    free(s->ws);
    s->ws = xcalloc((size_t)n + 1, sizeof(ws_item));
    for (int64_t i = 0; i < n; ++i) {
        s->ws[i].part = part[i]; s->ws[i].key = key[i];
        for (int k = 0; k < 3; ++k) s->ws[i].lam[k] = lam[3 * i + k];
    }
    qsort(s->ws, n, sizeof(ws_item), cmp_ws);
    s->ws_n = n;
}

int64_t orc_warmstart_size(const orc_sim *s) { return s->ws_n; }

void orc_get_warmstart(const orc_sim *s, int *part, uint64_t *key, double *lam) {
    for (int64_t i = 0; i < s->ws_n; ++i) {
        part[i] = s->ws[i].part; key[i] = s->ws[i].key;
        for (int k = 0; k < 3; ++k) lam[3 * i + k] = s->ws[i].lam[k];
    }
}

static const double *ws_lookup(const orc_sim *s, int part, uint64_t key) {
    ws_item probe;
    probe.part = part; probe.key = key;
    const ws_item *hit = bsearch(&probe, s->ws, s->ws_n, sizeof(ws_item), cmp_ws);
    return hit ? hit->lam : NULL;
}

/* ------------------------------------------------------------------------ */
/* c6: one worker's timestep -- PGS on the MLCP of Eq 1-7 over its active     */
/* bodies and constraints, then integration (Section 3: velocities first,     */
/* then positions with the new velocities).                                   */
/* ------------------------------------------------------------------------ */

/* Arithmetic type of the PGS arrays (velocities, impulses, row
 * coefficients).  FP64 is the oracle.  Built with -DORC_REAL=float, the same
 * algorithm in the same order runs its sweeps in FP32: a measure of how far
 * FP32 arithmetic alone can stay from the FP64 result on a given step (the
 * contact geometry, weights and blend stay FP64). */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

typedef struct {
    int la, lb;          /* local body indices, -1 = static end */
    real JA[6], JB[6];   /* (linear, angular) Jacobian blocks */
    real k;              /* 1 / (J M^-1 J^T) */
    real target;
    int friction_of;     /* row index of the normal row for friction rows, else -1 */
    real mu;
    int bilateral;       /* joint rows: bounds +-inf */
    int full;            /* a box end: angular response through its 3 x 3 inverse inertia */
    real IA[3], IB[3];   /* with full: Iw_A JA_ang, Iw_B JB_ang */
} pgs_row;

static void row_bounds(const pgs_row *r, const real *lam, real *lo, real *hi) {
    if (r->friction_of >= 0) {
        real ln = lam[r->friction_of];
        *lo = -r->mu * ln; *hi = r->mu * ln;
    } else if (r->bilateral) {
        *lo = -INFINITY; *hi = INFINITY;
    } else {
        *lo = 0.0; *hi = INFINITY;
    }
}

static real clampd(real x, real lo, real hi) { return x < lo ? lo : (x > hi ? hi : x); }

static real row_velocity(const pgs_row *r, const real *vel) {
    real w = 0;
    if (r->la >= 0) for (int a = 0; a < 6; ++a) w += r->JA[a] * vel[6 * r->la + a];
    if (r->lb >= 0) for (int a = 0; a < 6; ++a) w += r->JB[a] * vel[6 * r->lb + a];
    return w;
}

static void apply_impulse(const pgs_row *r, real *vel, const real *minv, real dl) {
    if (r->full) {
        if (r->la >= 0)
            for (int a = 0; a < 3; ++a) {
                vel[6 * r->la + a] += minv[6 * r->la + a] * r->JA[a] * dl;
                vel[6 * r->la + 3 + a] += r->IA[a] * dl;
            }
        if (r->lb >= 0)
            for (int a = 0; a < 3; ++a) {
                vel[6 * r->lb + a] += minv[6 * r->lb + a] * r->JB[a] * dl;
                vel[6 * r->lb + 3 + a] += r->IB[a] * dl;
            }
        return;
    }
    if (r->la >= 0) for (int a = 0; a < 6; ++a) vel[6 * r->la + a] += minv[6 * r->la + a] * r->JA[a] * dl;
    if (r->lb >= 0) for (int a = 0; a < 6; ++a) vel[6 * r->lb + a] += minv[6 * r->lb + a] * r->JB[a] * dl;
}

static double row_residual(const pgs_row *r, const real *vel, const real *lam, int i) {
    real lo, hi;
    row_bounds(r, lam, &lo, &hi);
    real w = row_velocity(r, vel);
    real proj = clampd(lam[i] + r->k * (r->target - w), lo, hi);
    return (lam[i] - proj) / r->k;
}

/* one row of a rigid constraint along direction d between lever arms rA, rB
 * (vectors from each body's centre to the constraint point) */
static void make_row(pgs_row *row, int la, int lb, const double d[3], const double rA[3],
                     const double rB[3], const real *minv) {
    double ca[3], cb[3];
    cross3(rA, d, ca);
    cross3(rB, d, cb);
    row->la = la; row->lb = lb;
    for (int a = 0; a < 3; ++a) {
        row->JA[a] = -d[a]; row->JA[3 + a] = -ca[a];
        row->JB[a] = d[a];  row->JB[3 + a] = cb[a];
    }
    double s = 0;
    if (la >= 0) for (int a = 0; a < 6; ++a) s += row->JA[a] * minv[6 * la + a] * row->JA[a];
    if (lb >= 0) for (int a = 0; a < 6; ++a) s += row->JB[a] * minv[6 * lb + a] * row->JB[a];
    row->k = 1.0 / s;
    row->friction_of = -1; row->bilateral = 0; row->mu = 0; row->target = 0;
    row->full = 0;
}

/* make_row with a box at either end: that end's angular response is its
 * world inverse inertia (Iw, row-major; NULL for a sphere, which keeps the
 * isotropic minv entries) applied to the angular Jacobian block */
static void make_row_full(pgs_row *row, int la, int lb, const double d[3], const double rA[3], const double rB[3],
                          const real *minv, const double *IwA, const double *IwB) {
    make_row(row, la, lb, d, rA, rB, minv);
    row->full = 1;
    double s = 0;
    for (int a = 0; a < 3; ++a) { row->IA[a] = 0; row->IB[a] = 0; }
    if (la >= 0) {
        for (int a = 0; a < 3; ++a) {
            s += row->JA[a] * minv[6 * la + a] * row->JA[a];
            row->IA[a] = IwA ? IwA[3 * a] * row->JA[3] + IwA[3 * a + 1] * row->JA[4] + IwA[3 * a + 2] * row->JA[5]
                             : minv[6 * la + 3 + a] * row->JA[3 + a];
        }
        for (int a = 0; a < 3; ++a) s += row->JA[3 + a] * row->IA[a];
    }
    if (lb >= 0) {
        for (int a = 0; a < 3; ++a) {
            s += row->JB[a] * minv[6 * lb + a] * row->JB[a];
            row->IB[a] = IwB ? IwB[3 * a] * row->JB[3] + IwB[3 * a + 1] * row->JB[4] + IwB[3 * a + 2] * row->JB[5]
                             : minv[6 * lb + 3 + a] * row->JB[3 + a];
        }
        for (int a = 0; a < 3; ++a) s += row->JB[3 + a] * row->IB[a];
    }
    row->k = 1.0 / s;
}

/* world inverse inertia of a solid box: R diag(1/I) R^T */
static void box_world_inv_inertia(const double q[4], const double h[3], double im, double Iw[9]) {
    double R[9], dI[3];
    quat_to_matrix(q, R);
    for (int k = 0; k < 3; ++k) {
        const double a = h[(k + 1) % 3], b = h[(k + 2) % 3];
        dI[k] = im > 0 ? 3.0 * im / (a * a + b * b) : 0.0;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Iw[3 * r + c] = R[3 * r] * dI[0] * R[3 * c] + R[3 * r + 1] * dI[1] * R[3 * c + 1] + R[3 * r + 2] * dI[2] * R[3 * c + 2];
}

typedef struct {
    int part;
    int64_t first_pair, n_pairs;
} worker_view;

static int local_index(const int *bodies, int nb, int b) {
    int lo = 0, hi = nb;
    while (lo < hi) { int mid = (lo + hi) / 2; if (bodies[mid] < b) lo = mid + 1; else hi = mid; }
    return (lo < nb && bodies[lo] == b) ? lo : -1;
}

static void solve_worker(orc_sim *s, int part, int scene, const int *bodies, int nb,
                         const int64_t *body_entry, int64_t p0, int64_t p1, double h_override,
                         int iters) {
    const orc_params *P = &s->P;
    double h = h_override > 0 ? h_override : s->dt[scene];
    double mu = s->mu[scene];
    real *vel = xcalloc((size_t)nb * 6 + 1, sizeof(real));
    real *minv = xcalloc((size_t)nb * 6 + 1, sizeof(real));
    for (int i = 0; i < nb; ++i) {
        int b = bodies[i];
        const double *x = s->st + 13 * (size_t)b;
        for (int a = 0; a < 3; ++a) {
            vel[6 * i + a] = x[7 + a] + h * P->gravity[a];   /* external force h*f */
            vel[6 * i + 3 + a] = x[10 + a];
            minv[6 * i + a] = s->im[b];
            minv[6 * i + 3 + a] = s->iI[b];
        }
    }
    /* box bodies: world inverse inertia from the blended orientation */
    double *iw = NULL;
    if (s->half) {
        iw = xcalloc((size_t)nb * 9 + 1, sizeof(double));
        for (int i = 0; i < nb; ++i)
            if (body_is_box(s, bodies[i]))
                box_world_inv_inertia(s->st + 13 * (size_t)bodies[i] + 3, s->half + 3 * (size_t)bodies[i],
                                      s->im[bodies[i]], iw + 9 * (size_t)i);
    }
#define IW_OF(l, body) ((l) >= 0 && iw && body_is_box(s, (body)) ? iw + 9 * (size_t)(l) : NULL)
    int64_t np_ = p1 - p0;
    pgs_row *rows = xcalloc((size_t)np_ * 3 + 1, sizeof(pgs_row));
    real *lam = xcalloc((size_t)np_ * 3 + 1, sizeof(real));
    int *slots = xcalloc((size_t)np_ * 2 + 1, sizeof(int));
    uint64_t *prio = xcalloc((size_t)np_ + 1, sizeof(uint64_t));
    /* rows, fixed for the step from the blended state (Alg 1) */
    for (int64_t q = 0; q < np_; ++q) {
        int64_t pi = p0 + q;
        pgs_row *r3 = rows + 3 * q;
        if (s->pair_kind[pi] == 0) {
            const orc_contact *c = &s->con[s->pair_cidx[pi]];
            int a = c->a, b = c->b;
            int la = (s->im[a] > 0) ? local_index(bodies, nb, a) : -1;
            int lb = (b < s->n && s->im[b] > 0) ? local_index(bodies, nb, b) : -1;
            double ra = s->rad[a];
            double rA[3] = {ra * c->n[0], ra * c->n[1], ra * c->n[2]};
            double rB[3] = {0, 0, 0};
            if (b < s->n) { double rb = s->rad[b]; for (int k = 0; k < 3; ++k) rB[k] = -rb * c->n[k]; }
            double t2[3];
            cross3(c->n, c->t1, t2);
            if (c->at_point) {
                /* box contact: both lever arms reach the contact point */
                const double *xa = s->st + 13 * (size_t)a;
                for (int k = 0; k < 3; ++k) rA[k] = c->p[k] - xa[k];
                if (b < s->n) {
                    const double *xb = s->st + 13 * (size_t)b;
                    for (int k = 0; k < 3; ++k) rB[k] = c->p[k] - xb[k];
                }
                const double *IwA = IW_OF(la, a), *IwB = b < s->n ? IW_OF(lb, b) : NULL;
                make_row_full(&r3[0], la, lb, c->n, rA, rB, minv, IwA, IwB);
                make_row_full(&r3[1], la, lb, c->t1, rA, rB, minv, IwA, IwB);
                make_row_full(&r3[2], la, lb, t2, rA, rB, minv, IwA, IwB);
            } else {
                make_row(&r3[0], la, lb, c->n, rA, rB, minv);
                make_row(&r3[1], la, lb, c->t1, rA, rB, minv);
                make_row(&r3[2], la, lb, t2, rA, rB, minv);
            }
            r3[0].target = c->phi > 0 ? -c->phi / h : P->erp * fmax(-c->phi - P->slop, 0.0) / h;
            r3[1].friction_of = (int)(3 * q); r3[1].mu = mu;
            r3[2].friction_of = (int)(3 * q); r3[2].mu = mu;
            slots[2 * q] = la; slots[2 * q + 1] = lb;
        } else {
            int j = (int)s->pair_cidx[pi];
            int a = s->jab[2 * j], b = s->jab[2 * j + 1];
            const double *anc = s->janc + 6 * (size_t)j;
            double pA[3], pB[3], rA[3] = {0, 0, 0}, rB[3] = {0, 0, 0};
            int la = -1, lb = -1;
            if (a >= 0) {
                const double *x = s->st + 13 * (size_t)a;
                double R[9];
                quat_to_matrix(x + 3, R);
                mat_vec(R, anc, rA);
                for (int k = 0; k < 3; ++k) pA[k] = x[k] + rA[k];
                if (s->im[a] > 0) la = local_index(bodies, nb, a);
            } else {
                for (int k = 0; k < 3; ++k) pA[k] = anc[k];
            }
            if (b >= 0) {
                const double *x = s->st + 13 * (size_t)b;
                double R[9];
                quat_to_matrix(x + 3, R);
                mat_vec(R, anc + 3, rB);
                for (int k = 0; k < 3; ++k) pB[k] = x[k] + rB[k];
                if (s->im[b] > 0) lb = local_index(bodies, nb, b);
            } else {
                for (int k = 0; k < 3; ++k) pB[k] = anc[3 + k];
            }
            const double *IwA = a >= 0 ? IW_OF(la, a) : NULL, *IwB = b >= 0 ? IW_OF(lb, b) : NULL;
            for (int ax = 0; ax < 3; ++ax) {
                double e[3] = {0, 0, 0};
                e[ax] = 1.0;
                if (IwA || IwB) make_row_full(&r3[ax], la, lb, e, rA, rB, minv, IwA, IwB);
                else make_row(&r3[ax], la, lb, e, rA, rB, minv);
                r3[ax].bilateral = 1;
                r3[ax].target = -P->erp * (pB[ax] - pA[ax]) / h;
            }
            slots[2 * q] = la; slots[2 * q + 1] = lb;
        }
        /* priority mix64(kind<<62 ^ key); pair_key already holds kind<<62 ^ key */
        prio[q] = orc_mix64(s->pair_key[pi]);
    }
    /* c5: greedy colouring in priority order */
    int *colour = xcalloc((size_t)np_ + 1, sizeof(int));
    int ncol = np_ > 0 ? colour_nodes((int)np_, slots, prio, nb, colour) : 0;
    if (ncol < 0) ncol = ORC_MAX_COLOURS;
    for (int64_t q = 0; q < np_; ++q) s->pair_colour[p0 + q] = colour[q];
    s->part_colours[part] = ncol;
    /* warm start: previous impulses of the same (worker, constraint) */
    for (int64_t q = 0; q < np_; ++q) {
        const double *prev = ws_lookup(s, part, s->pair_key[p0 + q]);
        for (int k = 0; k < 3; ++k) {
            real l0 = prev ? (real)(prev[k] * P->warmstart) : (real)0;
            lam[3 * q + k] = l0;
            if (l0 != 0.0) apply_impulse(&rows[3 * q + k], vel, minv, l0);
        }
    }
    /* constraints grouped by colour, canonical order inside a colour */
    int64_t *by_colour = xcalloc((size_t)np_ + 1, sizeof(int64_t));
    int64_t *col_start = xcalloc((size_t)ncol + 2, sizeof(int64_t));
    for (int64_t q = 0; q < np_; ++q) col_start[colour[q] + 1]++;
    for (int c = 0; c < ncol; ++c) col_start[c + 1] += col_start[c];
    {
        int64_t *fill = xcalloc((size_t)ncol + 1, sizeof(int64_t));
        for (int64_t q = 0; q < np_; ++q) by_colour[col_start[colour[q]] + fill[colour[q]]++] = q;
        free(fill);
    }
    /* sweeps: Gauss-Seidel with projection onto [lo, hi] (Eq 5-7) */
    int it_done = 0;
    for (int it = 0; it < iters; ++it) {
        for (int c = 0; c < ncol; ++c) {
            for (int64_t t = col_start[c]; t < col_start[c + 1]; ++t) {
                int64_t q = by_colour[t];
                for (int k = 0; k < 3; ++k) {
                    int i = (int)(3 * q + k);
                    const pgs_row *r = &rows[i];
                    real lo, hi;
                    row_bounds(r, lam, &lo, &hi);
                    real w = row_velocity(r, vel);
                    real lnew = clampd(lam[i] + r->k * (r->target - w), lo, hi);
                    real dl = lnew - lam[i];
                    lam[i] = lnew;
                    apply_impulse(r, vel, minv, dl);
                }
            }
        }
        it_done = it + 1;
        if (P->res_tol > 0 && P->res_check_every > 0 && it_done % P->res_check_every == 0 &&
            np_ > 0) {
            double sq = 0;
            for (int64_t i = 0; i < 3 * np_; ++i) { double rr = row_residual(&rows[i], vel, lam, (int)i); sq += rr * rr; }
            if (sqrt(sq / (double)(3 * np_)) <= P->res_tol) break;
        }
    }
    /* c10: residual at the final iterate */
    double sq = 0, rmax = 0;
    for (int64_t i = 0; i < 3 * np_; ++i) {
        double rr = row_residual(&rows[i], vel, lam, (int)i);
        sq += rr * rr;
        if (fabs(rr) > rmax) rmax = fabs(rr);
    }
    s->part_res_sq[part] = sq;
    s->part_res_max[part] = rmax;
    s->part_rows[part] = 3 * np_;
    s->part_iters[part] = it_done;
    for (int64_t q = 0; q < np_; ++q)
        for (int k = 0; k < 3; ++k) s->pair_lam[3 * (p0 + q) + k] = lam[3 * q + k];
    /* integrate: x += h v, q <- normalise(q + h/2 (0, w) (x) q); write this
     * worker's copy of every active body */
    for (int i = 0; i < nb; ++i) {
        int b = bodies[i];
        const double *x = s->st + 13 * (size_t)b;
        double *out = s->copies + 13 * (size_t)body_entry[i];
        double om[4] = {0, vel[6 * i + 3], vel[6 * i + 4], vel[6 * i + 5]};
        double dq[4];
        quat_mul(om, x + 3, dq);
        double qn[4];
        for (int a = 0; a < 4; ++a) qn[a] = x[3 + a] + 0.5 * h * dq[a];
        double L = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int a = 0; a < 3; ++a) out[a] = x[a] + h * vel[6 * i + a];
        for (int a = 0; a < 4; ++a) out[3 + a] = qn[a] / L;
        for (int a = 0; a < 3; ++a) { out[7 + a] = vel[6 * i + a]; out[10 + a] = vel[6 * i + 3 + a]; }
    }
    free(vel); free(minv); free(rows); free(lam); free(slots); free(prio); free(colour);
    free(by_colour); free(col_start); free(iw);
#undef IW_OF
}

/* ------------------------------------------------------------------------ */
/* Learned warm start: features of every (worker, contact) pair, read from   */
/* the blended state at the start of the step (definitions in the header).   */
/* ------------------------------------------------------------------------ */

static void compute_features(orc_sim *s, double dt_override) {
    const int n = s->n;
    /* depth: breadth-first from every body of O at once */
    s->depth = xcalloc((size_t)n + 1, 1);
    int *queue = xcalloc((size_t)n + 1, sizeof(int));
    int head = 0, tail = 0;
    for (int b = 0; b < n; ++b) {
        if (s->im[b] > 0 && popc64(s->mask[b]) >= 2) { s->depth[b] = 0; queue[tail++] = b; }
        else s->depth[b] = ORC_DEPTH_CAP;
    }
    while (head < tail) {
        int u = queue[head++];
        if (s->depth[u] + 1 >= ORC_DEPTH_CAP) continue;
        for (int k = s->row_ptr[u]; k < s->row_ptr[u + 1]; ++k) {
            int v = s->col[k];
            if (s->depth[v] != ORC_DEPTH_CAP) continue;
            s->depth[v] = (uint8_t)(s->depth[u] + 1);
            queue[tail++] = v;
        }
    }
    free(queue);
    double g = sqrt(dot3(s->P.gravity, s->P.gravity));
    double g_ref = g > 1.0 ? g : 1.0;
    s->pair_feat = xcalloc((size_t)s->npairs * ORC_NFEAT + 1, sizeof(double));
    s->pair_scale = xcalloc((size_t)s->npairs + 1, sizeof(double));
    s->pair_found = xcalloc((size_t)s->npairs + 1, sizeof(int));
    for (int64_t q = 0; q < s->npairs; ++q) {
        const double *prev = ws_lookup(s, s->pair_part[q], s->pair_key[q]);
        s->pair_found[q] = prev != NULL;
        if (s->pair_kind[q] != 0) continue;
        const orc_contact *c = &s->con[s->pair_cidx[q]];
        int a = c->a, b = c->b;
        int dyn_a = s->im[a] > 0, dyn_b = b < n && s->im[b] > 0;
        int scene = s->sob[a];
        double h = dt_override > 0 ? dt_override : s->dt[scene];
        /* velocity of each end's contact point; rA = r_a n, rB = -r_b n */
        double pa[3] = {0, 0, 0}, pb[3] = {0, 0, 0};
        if (dyn_a) {
            const double *x = s->st + 13 * (size_t)a;
            double rA[3] = {s->rad[a] * c->n[0], s->rad[a] * c->n[1], s->rad[a] * c->n[2]}, wr[3];
            cross3(x + 10, rA, wr);
            for (int k = 0; k < 3; ++k) pa[k] = x[7 + k] + wr[k];
        }
        if (dyn_b) {
            const double *x = s->st + 13 * (size_t)b;
            double rB[3] = {-s->rad[b] * c->n[0], -s->rad[b] * c->n[1], -s->rad[b] * c->n[2]}, wr[3];
            cross3(x + 10, rB, wr);
            for (int k = 0; k < 3; ++k) pb[k] = x[7 + k] + wr[k];
        }
        double rel[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        double t2[3];
        cross3(c->n, c->t1, t2);
        double ima = dyn_a ? s->im[a] : 0.0, imb = dyn_b ? s->im[b] : 0.0;
        double scale = g_ref * h / (ima + imb);
        double *f = s->pair_feat + (size_t)q * ORC_NFEAT;
        f[0] = dot3(c->n, rel) / (g_ref * h);
        f[1] = dot3(c->t1, rel) / (g_ref * h);
        f[2] = dot3(t2, rel) / (g_ref * h);
        f[3] = fmax(-c->phi, 0.0) / (g_ref * h * h);
        for (int k = 0; k < 3; ++k) f[4 + k] = prev ? prev[k] * s->P.warmstart / scale : 0.0;
        f[7] = ima;
        f[8] = imb;
        f[9] = dyn_a ? (s->row_ptr[a + 1] - s->row_ptr[a]) / 8.0 : 0.0;
        f[10] = dyn_b ? (s->row_ptr[b + 1] - s->row_ptr[b]) / 8.0 : 0.0;
        int d = ORC_DEPTH_CAP;
        if (dyn_a && s->depth[a] < d) d = s->depth[a];
        if (dyn_b && s->depth[b] < d) d = s->depth[b];
        f[11] = (double)d / ORC_DEPTH_CAP;
        s->pair_scale[q] = scale;
    }
}

/* ------------------------------------------------------------------------ */
/* One timestep of Alg 1.                                                    */
/* dt > 0 overrides every scene's dt.                                        */
/* ------------------------------------------------------------------------ */

int orc_step(orc_sim *s, double dt, int iters) {
    free_step_records(s);
    const int n = s->n;
    s->res_sq_total = 0; s->res_max = 0; s->res_rows = 0;
    /* contacts */
    contact_input in = {n, s->st, s->rad, s->im, s->np, s->planes, s->plane_scene, s->sob,
                        s->sflags, s->P.margin, s->half};
    s->nc = contacts_impl(&in, 1, &s->con);
    /* constraint graph G^t from contacts and joints */
    int64_t nedge = s->nc + s->nj;
    int *eu = xcalloc((size_t)nedge + 1, sizeof(int)), *ev = xcalloc((size_t)nedge + 1, sizeof(int));
    for (int64_t i = 0; i < s->nc; ++i) { eu[i] = s->con[i].a; ev[i] = s->con[i].b < n ? s->con[i].b : -1; }
    for (int j = 0; j < s->nj; ++j) { eu[s->nc + j] = s->jab[2 * j]; ev[s->nc + j] = s->jab[2 * j + 1]; }
    s->nadj = build_graph(n, s->im, nedge, eu, ev, &s->row_ptr, &s->col);
    free(eu); free(ev);
    /* LOADBALANCE over contacts between two dynamic bodies */
    {
        int64_t m = 0;
        int *ca = xcalloc((size_t)s->nc + 1, sizeof(int)), *cb = xcalloc((size_t)s->nc + 1, sizeof(int));
        for (int64_t i = 0; i < s->nc; ++i) {
            int a = s->con[i].a, b = s->con[i].b;
            if (b >= n || s->im[a] == 0 || s->im[b] == 0 || s->con[i].k != 0) continue;   /* one per body pair */
            ca[m] = a; cb[m] = b; ++m;
        }
        int do_deact = s->P.lb_deact_every > 0 && (s->step_index % s->P.lb_deact_every) == 0;
        int64_t *weight = NULL;
        if (s->P.lb_load == 1) {   /* 1 + contacts per body, every contact of the step */
            weight = xcalloc((size_t)n + 1, sizeof(int64_t));
            for (int b = 0; b < n; ++b) weight[b] = 1;
            for (int64_t i = 0; i < s->nc; ++i) {
                if (s->con[i].k != 0) continue;   /* a box manifold counts once */
                weight[s->con[i].a]++;
                if (s->con[i].b < n) weight[s->con[i].b]++;
            }
        }
        int64_t *count = counts_from_masks(n, s->mask, s->sob, s->part_base, s->n_parts, weight);
        membership mem = {s->mask, s->sob, s->part_base, count, weight};
        if (s->P.lb_activate || do_deact)
            load_balance_impl(&mem, n, s->row_ptr, s->col, m, ca, cb, s->sgamma, s->P.lb_activate, do_deact);
        free(count); free(weight); free(ca); free(cb);
    }
    for (int b = 0; b < n; ++b)
        if (s->im[b] > 0 && s->mask[b] == 0) return ORC_ERR_MEMBERSHIP;
    /* P_i and O (Eq 9-10): entries (body, worker), body-major */
    s->entry_ptr = xcalloc((size_t)n + 1, sizeof(int64_t));
    for (int b = 0; b < n; ++b) s->entry_ptr[b + 1] = s->entry_ptr[b] + popc64(s->mask[b]);
    s->ne = s->entry_ptr[n];
    s->entry_part = xcalloc((size_t)s->ne + 1, sizeof(int));
    for (int b = 0; b < n; ++b) {
        int64_t e = s->entry_ptr[b];
        for (int w = 0; w < 64; ++w)
            if (s->mask[b] >> w & 1u) s->entry_part[e++] = s->part_base[s->sob[b]] + w;
    }
    /* weights from D(o,i) on G^t */
    s->D = xcalloc((size_t)s->ne + 1, 1);
    geodesics_impl(n, s->mask, s->sob, s->sbeta, s->row_ptr, s->col, s->entry_ptr, s->D);
    s->weight = xcalloc((size_t)s->ne + 1, sizeof(double));
    for (int b = 0; b < n; ++b) {
        int64_t e0 = s->entry_ptr[b];
        int k = (int)(s->entry_ptr[b + 1] - e0);
        if (k == 1) s->weight[e0] = 1.0;
        else if (k > 1 && s->P.weights == 1) for (int i = 0; i < k; ++i) s->weight[e0 + i] = 1.0 / k;
        else if (k > 1) orc_weights(k, s->D + e0, s->weight + e0);
    }
    /* constraints of every worker: all dynamic ends active there; contacts
     * (canonical order) then joints (index order) */
    int64_t ncons = s->nc + s->nj;
    uint64_t *cons_mask = xcalloc((size_t)ncons + 1, sizeof(uint64_t));
    int *cons_scene = xcalloc((size_t)ncons + 1, sizeof(int));
    for (int64_t i = 0; i < s->nc; ++i) {
        int a = s->con[i].a, b = s->con[i].b;
        uint64_t m = ~(uint64_t)0;
        int any = 0;
        if (s->im[a] > 0) { m &= s->mask[a]; any = 1; }
        if (b < n && s->im[b] > 0) { m &= s->mask[b]; any = 1; }
        cons_mask[i] = any ? m : 0;
        cons_scene[i] = s->sob[a];
    }
    for (int j = 0; j < s->nj; ++j) {
        int a = s->jab[2 * j], b = s->jab[2 * j + 1];
        uint64_t m = ~(uint64_t)0;
        int any = 0;
        if (a >= 0 && s->im[a] > 0) { m &= s->mask[a]; any = 1; }
        if (b >= 0 && s->im[b] > 0) { m &= s->mask[b]; any = 1; }
        cons_mask[s->nc + j] = any ? m : 0;
        cons_scene[s->nc + j] = a >= 0 ? s->sob[a] : (b >= 0 ? s->sob[b] : 0);
    }
    int64_t *pcount = xcalloc((size_t)s->n_parts + 1, sizeof(int64_t));
    for (int64_t i = 0; i < ncons; ++i)
        for (int w = 0; w < 64; ++w)
            if (cons_mask[i] >> w & 1u) pcount[s->part_base[cons_scene[i]] + w]++;
    int64_t *pstart = xcalloc((size_t)s->n_parts + 2, sizeof(int64_t));
    for (int p = 0; p < s->n_parts; ++p) pstart[p + 1] = pstart[p] + pcount[p];
    s->npairs = pstart[s->n_parts];
    s->pair_part = xcalloc((size_t)s->npairs + 1, sizeof(int));
    s->pair_kind = xcalloc((size_t)s->npairs + 1, sizeof(int));
    s->pair_cidx = xcalloc((size_t)s->npairs + 1, sizeof(int64_t));
    s->pair_key = xcalloc((size_t)s->npairs + 1, sizeof(uint64_t));
    s->pair_colour = xcalloc((size_t)s->npairs + 1, sizeof(int));
    s->pair_lam = xcalloc((size_t)s->npairs * 3 + 1, sizeof(double));
    {
        int64_t *fill = xcalloc((size_t)s->n_parts + 1, sizeof(int64_t));
        for (int64_t i = 0; i < ncons; ++i)
            for (int w = 0; w < 64; ++w) {
                if (!(cons_mask[i] >> w & 1u)) continue;
                int p = s->part_base[cons_scene[i]] + w;
                int64_t q = pstart[p] + fill[p]++;
                s->pair_part[q] = p;
                if (i < s->nc) {
                    s->pair_kind[q] = 0;
                    s->pair_cidx[q] = i;
                    /* (a, b, k) packed so that key order is the canonical
                                     * contact order: a << 32 | b << 2 | k */
                    s->pair_key[q] = ((uint64_t)(uint32_t)s->con[i].a << 32) |
                                     ((uint64_t)(uint32_t)s->con[i].b << 2) | (uint64_t)(uint32_t)s->con[i].k;
                } else {
                    s->pair_kind[q] = 1;
                    s->pair_cidx[q] = i - s->nc;
                    s->pair_key[q] = ((uint64_t)1 << 62) | (uint64_t)(i - s->nc);
                }
            }
        free(fill);
    }
    free(cons_mask); free(cons_scene);
    compute_features(s, dt);
    /* every worker takes its timestep (sequentially here) */
    s->copies = xcalloc((size_t)s->ne * 13 + 1, sizeof(double));
    s->part_iters = xcalloc((size_t)s->n_parts + 1, sizeof(int));
    s->part_res_sq = xcalloc((size_t)s->n_parts + 1, sizeof(double));
    s->part_res_max = xcalloc((size_t)s->n_parts + 1, sizeof(double));
    s->part_rows = xcalloc((size_t)s->n_parts + 1, sizeof(int64_t));
    s->part_colours = xcalloc((size_t)s->n_parts + 1, sizeof(int));
    {
        /* bodies of each worker in ascending order, with their entry index */
        int64_t *bstart = xcalloc((size_t)s->n_parts + 2, sizeof(int64_t));
        for (int64_t e = 0; e < s->ne; ++e) bstart[s->entry_part[e] + 1]++;
        for (int p = 0; p < s->n_parts; ++p) bstart[p + 1] += bstart[p];
        int *pbody = xcalloc((size_t)s->ne + 1, sizeof(int));
        int64_t *pentry = xcalloc((size_t)s->ne + 1, sizeof(int64_t));
        int64_t *fill = xcalloc((size_t)s->n_parts + 1, sizeof(int64_t));
        for (int b = 0; b < n; ++b)
            for (int64_t e = s->entry_ptr[b]; e < s->entry_ptr[b + 1]; ++e) {
                int p = s->entry_part[e];
                int64_t k = bstart[p] + fill[p]++;
                pbody[k] = b; pentry[k] = e;
            }
        int *scene_of_part = xcalloc((size_t)s->n_parts + 1, sizeof(int));
        for (int p = 0, scene = 0; p < s->n_parts; ++p) {
            while (scene + 1 < s->ns && s->part_base[scene + 1] <= p) ++scene;
            scene_of_part[p] = scene;
        }
        /* workers write disjoint records (their pairs, entries and per-part
         * sums), so they may run on several threads with the same results */
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_thread_count())
        for (int p = 0; p < s->n_parts; ++p)
            solve_worker(s, p, scene_of_part[p], pbody + bstart[p], (int)(bstart[p + 1] - bstart[p]),
                         pentry + bstart[p], pstart[p], pstart[p + 1], dt, iters);
        /* residual totals in worker order */
        for (int p = 0; p < s->n_parts; ++p) {
            s->res_sq_total += s->part_res_sq[p];
            s->res_rows += s->part_rows[p];
            if (s->part_res_max[p] > s->res_max) s->res_max = s->part_res_max[p];
        }
        free(scene_of_part); free(bstart); free(pbody); free(pentry); free(fill);
    }
    free(pcount); free(pstart);
    /* blend overlap bodies; others take their single copy */
    for (int b = 0; b < n; ++b) {
        int64_t e0 = s->entry_ptr[b];
        int k = (int)(s->entry_ptr[b + 1] - e0);
        if (k == 0) {
            /* static body: unchanged */
        } else if (k == 1) {
            memcpy(s->st + 13 * (size_t)b, s->copies + 13 * (size_t)e0, 13 * sizeof(double));
        } else {
            orc_blend(k, s->copies + 13 * (size_t)e0, s->weight + e0, s->st + 13 * (size_t)b);
        }
    }
    /* joint error after the step (position level) */
    {
        double je[2];
        orc_joint_error(s, je);
        s->joint_violation_sum = je[0];
        s->joint_violation_max = je[1];
    }
    /* keep impulses for the next step's warm start */
    free(s->ws);
    s->ws = xcalloc((size_t)s->npairs + 1, sizeof(ws_item));
    for (int64_t q = 0; q < s->npairs; ++q) {
        s->ws[q].part = s->pair_part[q];
        s->ws[q].key = s->pair_key[q];
        for (int k = 0; k < 3; ++k) s->ws[q].lam[k] = s->pair_lam[3 * q + k];
    }
    qsort(s->ws, s->npairs, sizeof(ws_item), cmp_ws);
    s->ws_n = s->npairs;
    s->step_index++;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Read-back of the last step's records                                      */
/* ------------------------------------------------------------------------ */

/* counts: [contacts, adjacency length, entries, pairs, n_parts] */
void orc_get_counts(const orc_sim *s, int64_t *out) {
    out[0] = s->nc; out[1] = s->nadj; out[2] = s->ne; out[3] = s->npairs; out[4] = s->n_parts;
}

void orc_get_contacts(const orc_sim *s, int *ab, double *phi, double *nrm, double *t1) {
    for (int64_t i = 0; i < s->nc; ++i) {
        ab[2 * i] = s->con[i].a; ab[2 * i + 1] = s->con[i].b;
        phi[i] = s->con[i].phi;
        for (int k = 0; k < 3; ++k) { nrm[3 * i + k] = s->con[i].n[k]; t1[3 * i + k] = s->con[i].t1[k]; }
    }
}

/* manifold index and contact point of every contact (box contacts; the
 * point is zero for sphere contacts, whose rows use the radii) */
void orc_get_contact_points(const orc_sim *s, int *k, double *p) {
    for (int64_t i = 0; i < s->nc; ++i) {
        k[i] = s->con[i].k;
        for (int j = 0; j < 3; ++j) p[3 * i + j] = s->con[i].at_point ? s->con[i].p[j] : 0.0;
    }
}

/* per contact: how close the decisions of a box contact came to their
 * thresholds, in bands (< 1: a pair an FP32 computation may decide
 * otherwise); +inf for sphere contacts */
void orc_get_contact_amb(const orc_sim *s, double *amb) {
    for (int64_t i = 0; i < s->nc; ++i) amb[i] = s->con[i].amb;
}

void orc_get_graph(const orc_sim *s, int *row_ptr, int *col) {
    memcpy(row_ptr, s->row_ptr, ((size_t)s->n + 1) * sizeof(int));
    memcpy(col, s->col, (size_t)s->nadj * sizeof(int));
}

void orc_get_entries(const orc_sim *s, int64_t *entry_ptr, int *entry_part, uint8_t *D,
                     double *weight, double *copies) {
    memcpy(entry_ptr, s->entry_ptr, ((size_t)s->n + 1) * sizeof(int64_t));
    memcpy(entry_part, s->entry_part, (size_t)s->ne * sizeof(int));
    memcpy(D, s->D, (size_t)s->ne);
    memcpy(weight, s->weight, (size_t)s->ne * sizeof(double));
    memcpy(copies, s->copies, (size_t)s->ne * 13 * sizeof(double));
}

void orc_get_pairs(const orc_sim *s, int *part, int *kind, int64_t *cidx, uint64_t *key,
                   int *colour, double *lam) {
    memcpy(part, s->pair_part, (size_t)s->npairs * sizeof(int));
    memcpy(kind, s->pair_kind, (size_t)s->npairs * sizeof(int));
    memcpy(cidx, s->pair_cidx, (size_t)s->npairs * sizeof(int64_t));
    memcpy(key, s->pair_key, (size_t)s->npairs * sizeof(uint64_t));
    memcpy(colour, s->pair_colour, (size_t)s->npairs * sizeof(int));
    memcpy(lam, s->pair_lam, (size_t)s->npairs * 3 * sizeof(double));
}

/* per pair: ORC_NFEAT features, scale s, previous-impulse flag; per body:
 * depth to O (all of the last step) */
void orc_get_features(const orc_sim *s, double *feat, double *scale, int *found, uint8_t *depth) {
    memcpy(feat, s->pair_feat, (size_t)s->npairs * ORC_NFEAT * sizeof(double));
    memcpy(scale, s->pair_scale, (size_t)s->npairs * sizeof(double));
    memcpy(found, s->pair_found, (size_t)s->npairs * sizeof(int));
    memcpy(depth, s->depth, (size_t)s->n);
}

/* per worker: iterations run, residual sum of squares, rows, colours */
void orc_get_part_stats(const orc_sim *s, int *iters, double *res_sq, int64_t *rows, int *colours) {
    memcpy(iters, s->part_iters, (size_t)s->n_parts * sizeof(int));
    memcpy(res_sq, s->part_res_sq, (size_t)s->n_parts * sizeof(double));
    memcpy(rows, s->part_rows, (size_t)s->n_parts * sizeof(int64_t));
    memcpy(colours, s->part_colours, (size_t)s->n_parts * sizeof(int));
}

/* [rms residual over all rows of all workers, max |residual|, max joint gap,
 *  sum of joint gaps] after the last step */
void orc_get_metrics(const orc_sim *s, double *out) {
    out[0] = s->res_rows > 0 ? sqrt(s->res_sq_total / (double)s->res_rows) : 0.0;
    out[1] = s->res_max;
    out[2] = s->joint_violation_max;
    out[3] = s->joint_violation_sum;
}

void orc_joint_error(const orc_sim *s, double *out) {
    out[0] = 0.0;
    out[1] = 0.0;
    for (int j = 0; j < s->nj; ++j) {
        int a = s->jab[2 * j], b = s->jab[2 * j + 1];
        const double *anc = s->janc + 6 * (size_t)j;
        double pA[3], pB[3], r[3], R[9];
        if (a >= 0) {
            const double *x = s->st + 13 * (size_t)a;
            quat_to_matrix(x + 3, R);
            mat_vec(R, anc, r);
            for (int k = 0; k < 3; ++k) pA[k] = x[k] + r[k];
        } else {
            for (int k = 0; k < 3; ++k) pA[k] = anc[k];
        }
        if (b >= 0) {
            const double *x = s->st + 13 * (size_t)b;
            quat_to_matrix(x + 3, R);
            mat_vec(R, anc + 3, r);
            for (int k = 0; k < 3; ++k) pB[k] = x[k] + r[k];
        } else {
            for (int k = 0; k < 3; ++k) pB[k] = anc[3 + k];
        }
        double d[3] = {pB[0] - pA[0], pB[1] - pA[1], pB[2] - pA[2]};
        double L = sqrt(dot3(d, d));
        out[0] += L;
        if (L > out[1]) out[1] = L;
    }
}
