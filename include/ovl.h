/*
 * ovl.h -- C ABI of libovl, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of Kale & Kry, "Distributed Simulation of Large
 * Multi-body Systems" (overlapping-partition rigid-body simulation).
 *
 * In the paper N workers each simulate an overlapping subset P_i of the
 * bodies (Section 4, Eq 9-10) and a server blends the states of the shared
 * bodies O (Algorithm 1).  Here every worker is a partition solved by its own
 * CTA on one GPU; one call to ovl_step runs one timestep of Algorithm 1.
 *
 * Conventions
 *  - Every function returns ovl_status: 0 on success, a negative OVL_ERR_*
 *    code on failure; ovl_last_error(ctx) then gives a message.  No C++
 *    exception crosses this boundary.
 *  - Host arrays passed in are owned by the caller and only read during the
 *    call.  Device memory is owned by the library.  Arguments documented as
 *    "device pointer" take any CUDA device address (e.g. a torch tensor's
 *    data_ptr()) on the context's device.
 *  - A context is not thread-safe.  All work runs on the context's stream;
 *    ovl_read_* calls with host outputs synchronise that stream.
 *  - Body state layout (Eq 8): 13 floats per body, position x (3),
 *    quaternion q = (w, x, y, z) (4), linear velocity (3), angular
 *    velocity (3), world frame, row-major [n][13].
 *  - Workers: each scene has n_sets[s] <= 64 workers; a body's membership is
 *    a 64-bit mask W_b (bit w = scene-local worker w).  The global index of
 *    worker w of scene s is sum(n_sets[0..s-1]) + w.
 */
#ifndef OVL_H
#define OVL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ovl_status;

#define OVL_OK 0
#define OVL_ERR_ARG (-1)        /* bad argument or call order */
#define OVL_ERR_CUDA (-2)       /* a CUDA call failed */
#define OVL_ERR_CAPACITY (-3)   /* a fixed limit was exceeded: colours > 128 in a worker, sphere
                                   neighbours beyond a body's capacity (set from the radii), ... */
#define OVL_ERR_TIMEOUT (-4)    /* a bounded device-side wait gave up */
#define OVL_ERR_NONFINITE (-5)  /* NaN or Inf in a state */
#define OVL_ERR_MEMBERSHIP (-6) /* dynamic body with empty W, or a worker index >= n_sets */

typedef struct ovl_ctx ovl_ctx;

/* Method parameters (Section 3 constraint model; readings where the paper is
 * silent are marked). */
typedef struct ovl_params {
    float gravity[3];        /* external acceleration f/m, default (0,0,-9.81) */
    float margin;            /* contact when the gap phi <= margin, default 0.05 (reading) */
    float erp;               /* share of penetration / joint error removed per step, 0.2 (reading) */
    float slop;              /* penetration tolerated before push-out, 0.001 (reading) */
    float warmstart;         /* factor on the previous step's impulses, 1.0 */
    int32_t lb_activate;     /* 1: Algorithm 6's activation branch runs every step */
    int32_t lb_deact_every;  /* k > 0: Algorithm 6's removal branches on steps with index % k == 0; 0: never */
    float res_tol;           /* > 0: a worker stops sweeping once its RMS residual <= res_tol */
    int32_t res_check_every; /* sweeps between residual checks when res_tol > 0 */
    int32_t pgs_threads;     /* threads per worker CTA (0 = automatic) */
    int32_t flags;           /* OVL_FLAG_* */
    int32_t pgs_cluster;     /* CTAs per worker, 1, 2 or 4 (0 = automatic from the SM count) */
    int32_t smem_slot_limit; /* > 0: at most this many bodies per CTA in shared memory (larger
                                workers use the global-memory path); 0 = as many as fit */
    int32_t lb_load;         /* the load <W_x> Algorithm 6 compares: OVL_LB_BODIES (default) or
                                OVL_LB_CONTACTS; any other value is OVL_ERR_ARG at ovl_create */
    int32_t weights;         /* blending weights of overlap bodies: OVL_WEIGHTS_GEODESIC (default)
                                or OVL_WEIGHTS_UNIFORM; any other value is OVL_ERR_ARG */
} ovl_params;

/* Blending weights (Section 5.3).  GEODESIC is the method's: Eq 15 weights
 * proportional to 1 / D(o,i) of Eq 16.  UNIFORM is the naive choice the
 * paper compares against (Figure 8): every worker of an overlap body weighs
 * 1 / |W_b|.  The geodesic distances are computed (and readable) either way. */
#define OVL_WEIGHTS_GEODESIC 0
#define OVL_WEIGHTS_UNIFORM 1

/* Loads of Algorithm 6.  BODIES is the paper's: <W_x> counts the active
 * bodies of the workers in W_x (Table 1).  CONTACTS is the contact-following
 * load Section 6 proposes for scenes whose bodies carry very different
 * numbers of contacts: every active body counts 1 + the number of this
 * step's contacts it is an end of (planes and static ends included). */
#define OVL_LB_BODIES 0
#define OVL_LB_CONTACTS 1

#define OVL_FLAG_RESIDUAL 1  /* compute the complementarity residual of every row after the sweeps */
#define OVL_FLAG_TIMING 2    /* record per-phase times with CUDA events (ovl_read_stats) */
#define OVL_FLAG_AUTOTUNE 4  /* time the solver's launch shapes on the first step of every problem-size
                                bucket and keep the fastest (results are bit-identical across shapes) */
#define OVL_FLAG_FEATURES 8  /* compute the learned warm start's contact features every step, even
                                with the plain warm start (ovl_read_features) */

/* Warm-start modes (ovl_set_warmstart_mode).  PREVIOUS is the method's own
 * warm start: each (worker, constraint) starts from the impulses it had in
 * the previous step, times ovl_params.warmstart, or from zero.  The MLP
 * modes replace that start for contacts by the network's proposal (below);
 * joints always keep the previous impulses. */
#define OVL_WS_PREVIOUS 0
#define OVL_WS_MLP 1       /* every contact starts from the network's proposal */
#define OVL_WS_MLP_NEW 2   /* only contacts without previous impulses do */

/* A scene (or a batch of independent scenes whose bodies are contiguous). */
typedef struct ovl_scene_desc {
    int32_t n_bodies;
    const float *state;          /* [n][13] initial state */
    const float *radius;         /* [n] sphere radii (> 0) */
    const float *inv_mass;       /* [n] inverse masses; 0 = static body */
    int32_t n_planes;
    const float *planes;         /* [n_planes][4] (nx,ny,nz,d): plane n.p = d, free side n.p >= d; n unit */
    const int32_t *plane_scene;  /* [n_planes] scene of each plane, or NULL (all scene 0) */
    int32_t n_joints;
    const int32_t *joint_bodies; /* [n_joints][2] ball joints (a, b); -1 = world */
    const float *joint_anchors;  /* [n_joints][6] pivot in a's frame, pivot in b's frame (world if -1) */
    int32_t n_scenes;
    const int32_t *scene_of_body;/* [n] non-decreasing scene index, or NULL (all scene 0) */
    const float *scene_mu;       /* [n_scenes] Coulomb friction coefficient */
    const float *scene_dt;       /* [n_scenes] timestep h */
    const int32_t *scene_flags;  /* [n_scenes] bit 0: sphere-sphere contacts enabled */
    const int32_t *scene_gamma;  /* [n_scenes] overlap growth depth gamma (Alg 3, Alg 6) */
    const int32_t *scene_beta;   /* [n_scenes] weight search depth beta (Alg 5), <= 254 */
    const int32_t *n_sets;       /* [n_scenes] workers per scene, 1..64 */
    const float *half_extents;   /* [n][3] box half extents (zeros: a sphere), or NULL: all spheres.
                                    Finite and >= 0; a body with a positive extent is a solid box
                                    (inertia I_k = m (h_j^2 + h_l^2) / 3) whose radius must bound it
                                    (radius >= |h|: the broad phase tests bounding spheres).  Boxes
                                    are the bodies of the paper's Building and Bridge scenes
                                    (Section 6).  The learned warm start's contact features treat
                                    every contact as a sphere contact. */
} ovl_scene_desc;

/* Last-step statistics. */
typedef struct ovl_stats {
    int64_t n_contacts;        /* contacts of the last step (Alg 1) */
    int64_t n_adjacency;       /* directed adjacency entries of G^t (2 x edges) */
    int64_t n_entries;         /* sum over bodies of |W_b| */
    int64_t n_pairs;           /* (worker, constraint) pairs solved */
    int64_t n_rows;            /* PGS rows solved (3 per pair) */
    int64_t n_overlap;         /* |O| */
    int32_t n_workers;         /* total workers */
    int32_t max_colours;       /* largest colour count of any worker */
    int32_t max_iters;         /* most sweeps any worker ran */
    int32_t device_status;     /* first device-side error code of the step, 0 if none */
    double residual_rms;       /* RMS complementarity residual over all rows (OVL_FLAG_RESIDUAL) */
    double residual_max;       /* max |residual| */
    float phase_ms[12];        /* per-phase device times (OVL_FLAG_TIMING); see ovl_phase_name;
                                  index 10 = learned warm start (features + network), which the
                                  membership phase (index 3) includes; index 7 (geodesics) runs on
                                  its own stream beside the colouring and the solve when the
                                  workers do not outnumber the SMs, and the phases then add up to
                                  more than the total (index 9) */
    int64_t n_launches;        /* CUDA kernels the library launched during the last step */
    int32_t solve_cluster;     /* CTAs per worker of the last solve */
    int32_t solve_threads;     /* threads per CTA of the last solve */
    int32_t solve_rows_per_thread; /* rows a thread takes at once in a colour (colour block) */
    int32_t colour_rounds_max; /* most colouring rounds any worker needed */
    int64_t lb_candidates;     /* contacts handed to the host load balance in the last step */
    double lb_host_ms;         /* host time of the load balance in the last step (copies included) */
    int64_t solve_ctas;        /* CTAs the last solve launched */
    int64_t solve_ctas_masses; /* of those, CTAs holding the inverse masses in shared memory (two-record
                                  contact rows) */
} ovl_stats;

/* Fills *p with the defaults listed in ovl_params. */
ovl_status ovl_default_params(ovl_params *p);

/* Creates a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * to run on, or NULL for a stream the context owns.  *out receives the
 * context; destroy it with ovl_destroy.  The context also creates seven side
 * streams: six for concurrent per-class launches (priorities falling in
 * launch order) and one for the geodesic weights.  It sets the environment
 * variable CUDA_DEVICE_MAX_CONNECTIONS to 32 when it is unset, so that those
 * streams get hardware queues of their own.  That takes effect only if the
 * process has not yet created its CUDA context; otherwise, set the variable
 * before the first CUDA call. */
ovl_status ovl_create(ovl_ctx **out, const ovl_params *p, void *cuda_stream);
/* Frees the context's device and host memory, streams and events (after
 * finishing its work); NULL is OVL_ERR_ARG. */
ovl_status ovl_destroy(ovl_ctx *ctx);
/* Message of the context's last failed call (empty when none; "null
 * context" for NULL); the string belongs to the context and lives until
 * its next failing call. */
const char *ovl_last_error(const ovl_ctx *ctx);
/* Name of entry `phase` of ovl_stats.phase_ms (a static string; empty out
 * of range). */
const char *ovl_phase_name(int32_t phase);

/* Copies a scene to the device (Section 4: all bodies are loaded into every
 * worker's memory).  Replaces any previous scene, resets membership to empty,
 * the warm-start cache to empty and the step index to 0. */
ovl_status ovl_scene_upload(ovl_ctx *ctx, const ovl_scene_desc *scene);

/* Initial partitioning (Section 5.1 "semantic partitioning", Section 5.4
 * "naive division"): set_of_body[b] is b's single worker (scene-local).
 * Static bodies are ignored.  OVL_ERR_MEMBERSHIP if an index is out of range. */
ovl_status ovl_set_partition(ovl_ctx *ctx, const int32_t *set_of_body);

/* Sets every membership mask W_b directly ([n] host array); static bodies
 * must have 0, dynamic bodies a non-empty mask within their scene's workers. */
ovl_status ovl_set_membership(ovl_ctx *ctx, const uint64_t *masks);
ovl_status ovl_read_membership(ovl_ctx *ctx, uint64_t *masks);

/* ASSIGNTOOVERLAPSET (Algorithm 2 with GROWOVERLAP, Algorithm 3) over the
 * scene's joints in index order, on the joint graph, with each scene's
 * gamma.  Runs on the host (a setup step). */
ovl_status ovl_assign_overlap(ovl_ctx *ctx);

/* Blended state s^t (Eq 8).  on_device != 0: the pointer is a device
 * pointer, otherwise host memory; [n][13] floats. */
ovl_status ovl_set_state(ovl_ctx *ctx, const float *state13, int32_t on_device);
ovl_status ovl_read_state(ovl_ctx *ctx, float *state13, int32_t on_device);

/* Step counter used for the removal cadence of Algorithm 6. */
ovl_status ovl_set_step_index(ovl_ctx *ctx, int64_t step_index);

/* Warm-start cache: n entries (global worker, key, lambda[3]); key is
 * a<<32|b for a contact between bodies a < b (b = n_bodies + plane index for
 * a plane) and 1<<62 | j for joint j.  Replaces the cache. */
ovl_status ovl_set_warmstart(ovl_ctx *ctx, int64_t n, const int32_t *part, const uint64_t *key,
                             const float *lambda3);
/* Reads up to cap entries of the cache, sorted by (worker, key); *n gets the size. */
ovl_status ovl_read_warmstart(ovl_ctx *ctx, int64_t cap, int64_t *n, int32_t *part, uint64_t *key,
                              float *lambda3);

/* One timestep of Algorithm 1: contacts, constraint graph G^t, LOADBALANCE
 * (Algorithm 6), every worker's PGS solve of Eq 1-7 and integration, the
 * weights (Algorithm 5, Eq 15-16) and the blend (Algorithm 4).  dt > 0
 * overrides every scene's timestep; iters = PGS sweeps per worker. */
ovl_status ovl_step(ovl_ctx *ctx, float dt, int32_t iters);

/* Position-level joint violation of the current blended state (the error
 * measure of Section 6 for jointed scenes): for every ball joint the gap
 * |p_B - p_A| between its two pivots, p = x + R(q) anchor for a body end and
 * the anchor itself for a world end.  *sum gets the sum over all joints,
 * *max_gap the largest gap (metres); either pointer may be NULL.  FP32 gaps,
 * summed in FP64 in a fixed order (the result does not depend on timing).
 * Synchronises the context's stream. */
ovl_status ovl_joint_error(ovl_ctx *ctx, double *sum, double *max_gap);

/* ---- host-only entry points (no context, no CUDA call) -------------------
 * The library's own host implementations of the membership algorithms, run
 * on caller-supplied arrays; a step runs the same code after reading its
 * contacts back from the device.  Scenes are contiguous body ranges:
 * scene_of_body[n] is non-decreasing with values in [0, n_scenes); scene s
 * has n_sets[s] workers (1..64) and growth depth scene_gamma[s] >= 0.
 * mask[n] (in/out): bit w of mask[b] = body b active in worker w of its
 * scene; bits at or above the scene's n_sets give OVL_ERR_MEMBERSHIP.  Any
 * other malformed input gives OVL_ERR_ARG and leaves mask unchanged.  The
 * caller owns every array. */

/* LOADBALANCE (Algorithm 6, Section 5.4) with BRIDGE (Algorithm 7).
 * row_ptr[n + 1], col: CSR of the constraint graph G^t (edges inside one
 * scene).  contact_bodies[2 n_contacts]: the candidate contacts (a, b), in
 * the order they are processed (the step uses canonical order: ascending
 * (a, b), dynamic ends only); scenes must appear in ascending order.
 * contact_count[n]: NULL counts every active body once in the loads <W>
 * (Table 1); else body b counts 1 + contact_count[b] (the contact load).
 * do_activate / do_deactivate select the activation and the removal
 * branches.  threads (1..64): whole scenes go to up to that many host
 * threads; the result is the sequential one. */
ovl_status ovl_host_load_balance(int32_t n, const int32_t *scene_of_body, int32_t n_scenes,
                                 const int32_t *n_sets, const int32_t *scene_gamma, uint64_t *mask,
                                 const int32_t *row_ptr, const int32_t *col, int64_t n_contacts,
                                 const int32_t *contact_bodies, const int32_t *contact_count,
                                 int32_t do_activate, int32_t do_deactivate, int32_t threads);

/* ASSIGNTOOVERLAPSET (Algorithm 2) and GROWOVERLAP (Algorithm 3, Section
 * 5.1) over the joints in index order: a joint between two dynamic bodies
 * (inv_mass > 0) of different single workers makes each end active in the
 * other's worker and grows the overlap to depth gamma over the articulated
 * structure.  joint_bodies[2 n_joints]: body indices, -1 for the world. */
ovl_status ovl_host_assign_overlap(int32_t n, const int32_t *scene_of_body, int32_t n_scenes,
                                   const int32_t *n_sets, const int32_t *scene_gamma,
                                   const float *inv_mass, int32_t n_joints,
                                   const int32_t *joint_bodies, uint64_t *mask);

/* ---- box contact geometry (no context) -----------------------------------
 * Contacts of the box bodies of the paper's Building and Bridge scenes
 * (Section 6), one pair per index, computed by the library's FP32 contact
 * functions: on the GPU (on_gpu != 0: one thread per pair; the inputs are
 * copied to the device and the results back) or with the same functions on
 * the host (on_gpu == 0: no CUDA call).  Both runs give the same bits.  All
 * arrays are host arrays the caller owns.  A box is pose[7] = (x, y, z, qw,
 * qx, qy, qz) (unit quaternion) and half[3] (half extents).  The normal
 * points from the first shape towards the second; a gap is positive when
 * apart; a contact when gap <= margin.  Outputs per pair i: count[i] (0..4),
 * points[i][4][3] and gaps[i][4] (the first count[i] entries; the rest
 * zero), normal[i][3].  The step does not use these contacts yet.
 * n < 0 or a NULL array with n > 0 is OVL_ERR_ARG; a CUDA failure
 * OVL_ERR_CUDA. */

/* Box (first) against the plane n.x = d, plane[i] = (n, d) with n unit out
 * of the solid: the box's vertices within the margin, the 4 deepest (ties to
 * the lower vertex index, vertex v at (+-h0, +-h1, +-h2) by bits 0-2 of v).
 * normal = -n. */
ovl_status ovl_box_plane_contacts(int32_t n, const float *pose, const float *half, const float *plane,
                                  float margin, int32_t on_gpu, int32_t *count, float *points, float *gaps,
                                  float *normal);

/* Sphere (first; sphere[i] = (centre, radius)) against a box (second): the
 * box point nearest the centre, or with the centre inside the box its
 * projection on the face of least penetration.  gaps[i][0] holds the gap
 * even when count[i] == 0. */
ovl_status ovl_sphere_box_contacts(int32_t n, const float *sphere, const float *pose, const float *half,
                                   float margin, int32_t on_gpu, int32_t *count, float *points, float *gaps,
                                   float *normal);

/* Box A (first) against box B (second): the separating-axis test over the
 * 15 candidate axes; axis[i] = the chosen one (0-2 A's faces, 3-5 B's, 6 +
 * 3 i + j for a_i x b_j) or -1 when an axis separates them by more than the
 * margin.  A face axis gives the incident face clipped against the
 * reference face's sides (the 4 deepest points); an edge axis one point
 * midway between the supporting edges.  An edge axis is chosen over the best
 * face axis only when its separation exceeds 0.95 x the face's + 0.01 x the
 * smallest half extent. */
ovl_status ovl_box_box_contacts(int32_t n, const float *pose_a, const float *half_a, const float *pose_b,
                                const float *half_b, float margin, int32_t on_gpu, int32_t *count,
                                float *points, float *gaps, float *normal, int32_t *axis);

/* All contacts of a scene with box bodies (Algorithm 1's contact step for
 * row f1), in canonical order: every body a, then b > a of its scene
 * (pairs with scene_flags bit 0), then its scene's planes (b = n + plane),
 * and for a box manifold its points k = 0..3.  A pair is tested when its
 * bounding spheres (radius[]) meet in FP32, ((dx dx + dy dy) + dz dz) <=
 * ((ra + rb) + margin)^2 (a plane: ((n.p) - d) - r <= margin), the same
 * decision the sphere contacts take; then the box functions above decide
 * (two spheres: one contact, gap |d| - ra - rb).  Pairs of two static
 * bodies and planes of static bodies are skipped.  state13[n][13] (x, q, v,
 * w), radius[n], inv_mass[n], half[n][3] (zeros: a sphere),
 * scene_of_body[n], scene_flags[n_scenes], planes[n_planes][4],
 * plane_scene[n_planes].  Outputs, up to cap contacts: ab[][2], k[], phi[],
 * normal[][3] (from a towards b), point[][3]; *total = the number found
 * (more than cap: OVL_ERR_CAPACITY, the lists unwritten).  A brute-force
 * pair search: for tests and modest scenes.  GPU and host runs give the
 * same bits. */
ovl_status ovl_box_scene_contacts(int32_t n, const float *state13, const float *radius, const float *inv_mass,
                                  const float *half, const int32_t *scene_of_body, int32_t n_scenes,
                                  const int32_t *scene_flags, int32_t n_planes, const float *planes,
                                  const int32_t *plane_scene, float margin, int32_t on_gpu, int64_t cap,
                                  int64_t *total, int32_t *ab, int32_t *k, float *phi, float *normal,
                                  float *point);

/* Box rows (the solve of Eq 1-7 with a box's general lever arms and full
 * world inverse inertia R diag(1/I) R^T, I_k = m/3 (h_j^2 + h_l^2)): one
 * velocity step of each of n independent boxes on its own static plane.  v
 * += dt gravity, then `iters` Gauss-Seidel sweeps over the rows (normal, t1,
 * t2) of every ovl_box_plane_contacts contact in order: row d at lever r
 * has w = -d.v - (r x d).omega and k = 1 / (1/m + (r x d).Iw (r x d)); the
 * box takes -d (lambda' - lambda).  Normal bounds [0, inf), target -phi/dt
 * when phi > 0 else erp max(-phi - slop, 0)/dt; tangents within +-mu
 * lambda_n (current); t1 = normalise(e_k - n_k n) for the axis k of the
 * smallest |n_k|, t2 = n x t1.  inv_mass[n]; vel[n][6] = (v, omega) in and
 * out; count[n]; lam[n][12] = (n, t1, t2) impulses per contact (zero past
 * count).  On the GPU one thread per box, else the same functions on the
 * host; both give the same bits.  OVL_ERR_ARG / OVL_ERR_CUDA as above. */
ovl_status ovl_box_plane_step(int32_t n, const float *pose, const float *half, const float *inv_mass,
                              const float *plane, float mu, float dt, const float *gravity, float erp, float slop,
                              float margin, int32_t iters, int32_t on_gpu, float *vel, int32_t *count, float *lam);

/* LOADBALANCE (Algorithm 6 with BRIDGE, Algorithm 7) alone on the contacts
 * of the current state.  flags bit 0: activation branch, bit 1: removal
 * branches. */
ovl_status ovl_load_balance(ovl_ctx *ctx, int32_t flags);

/* Waits for all work of the context. */
ovl_status ovl_sync(ovl_ctx *ctx);

/* Records of the last step (host outputs, sized from ovl_read_stats):
 *  contacts: ab [m][2] (a < b; b >= n_bodies is a plane), phi [m], normal
 *            [m][3] (from a towards b), t1 [m][3]; canonical (a, b) order.
 *  graph:    row_ptr [n+1], col [n_adjacency], sorted and deduplicated.
 *  entries:  entry_ptr [n+1]; per entry (bodies in order, workers ascending):
 *            global worker, D(o,i) (255 = not met within beta, also for
 *            bodies outside O), weight, and the worker's copy [13].
 *  pairs:    per (worker, constraint) in (worker, key) order: worker, key,
 *            colour, lambda[3] after the sweeps. */
ovl_status ovl_read_stats(ovl_ctx *ctx, ovl_stats *out);
ovl_status ovl_read_contacts(ovl_ctx *ctx, int32_t *ab, float *phi, float *normal, float *t1);
/* Box contacts of the last step (the manifolds of Section 6's box bodies):
 * per contact its point index k in the pair's manifold (0..3; 0 for sphere
 * contacts) and its point [3] (zeros for sphere contacts).  Host arrays of
 * n_contacts entries (either may be NULL); OVL_ERR_ARG before a step. */
ovl_status ovl_read_contact_points(ovl_ctx *ctx, int32_t *k, float *point);
ovl_status ovl_read_graph(ovl_ctx *ctx, int32_t *row_ptr, int32_t *col);
ovl_status ovl_read_entries(ovl_ctx *ctx, int32_t *entry_ptr, int32_t *part, uint8_t *D,
                            float *weight, float *copies13);
ovl_status ovl_read_pairs(ovl_ctx *ctx, int32_t *part, uint64_t *key, int32_t *colour,
                          float *lambda3);
/* Autotuner cache (OVL_FLAG_AUTOTUNE) as JSON text, one entry per problem-size
 * bucket: {"P64_nb16384_q65536": {"cluster": 2, "threads": 512, "rows_per_thread": 2, "ms": 3.9}}.
 * export: writes at most cap bytes (NUL-terminated) and the full length to *len.
 * import: merges entries produced by export.  No counterpart in the paper:
 * this is the launch-shape tuner of the GPU solver. */
ovl_status ovl_autotune_export(ovl_ctx *ctx, char *buf, size_t cap, size_t *len);
ovl_status ovl_autotune_import(ovl_ctx *ctx, const char *json);

/* nsteps timesteps, as nsteps calls of ovl_step with the same dt and iters
 * (Algorithm 1's loop over t).  Each step reads a few counts back to size its
 * buffers and runs Algorithm 6 on the host, so the steps are issued one after
 * another from the host, not captured as one graph.  *done (optional)
 * receives the number of steps completed; the first failing step's status is
 * returned and the state is that of the last completed step. */
ovl_status ovl_step_n(ovl_ctx *ctx, float dt, int32_t iters, int32_t nsteps, int32_t *done);

/* Checkpoint of what a step reads (the paper's get/reset of a worker's state,
 * Section 4 and Table 1, for the whole simulation): the blended body state,
 * every mask W_b, the warm-start cache, the step index (Algorithm 6's
 * removal cadence), the warm-start mode, the network parameters with Adam's
 * moments (when set) and the autotuner's table.  Scene arrays are not in it.
 *
 * ovl_save: *len receives the checkpoint's size in bytes; with buf != NULL
 *   and cap >= *len the checkpoint is written to buf (host memory, caller-
 *   owned), else OVL_ERR_CAPACITY.  buf = NULL asks only for the size.
 *   Synchronises the context's stream.
 * ovl_load: restores a checkpoint into a context whose uploaded scene is the
 *   one it was saved from (same sizes and the same host arrays, checked by a
 *   hash; OVL_ERR_ARG otherwise, or when the bytes are not a checkpoint of
 *   this version).  Continuing from a load computes the same bits as
 *   continuing the saved run.  Records of the last step (ovl_read_contacts
 *   and the other per-step reads) are unavailable until the next step. */
ovl_status ovl_save(ovl_ctx *ctx, void *buf, size_t cap, size_t *len);
ovl_status ovl_load(ovl_ctx *ctx, const void *buf, size_t len);

/* Per worker: sweeps run, residual sum of squares, rows, colours. */
ovl_status ovl_read_worker_stats(ovl_ctx *ctx, int32_t *iters, double *res_sq, int64_t *rows,
                                 int32_t *colours);

/* The launch plan of the last step's solve (no counterpart in the paper: the
 * paper's workers are processes).  ctas [n_workers] (host, caller-owned):
 * how many CTAs, one thread-block cluster, solved each worker.  Every plan
 * computes the same bits; the plan changes only the time.  OVL_ERR_ARG before
 * the first step. */
ovl_status ovl_read_solve_plan(ovl_ctx *ctx, int32_t *ctas);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper)
 *
 * A 12-64-64-3 ReLU network proposes each contact's three impulses
 * (normal, t1, t2) from 12 features of the contact, all read from the
 * blended state at the start of the step, before gravity.  With
 * g_ref = max(|gravity|, 1) and s = g_ref h / (im_A + im_B) over the dynamic
 * ends (the impulse that cancels one step of gravity on the normal row):
 *   0-2  J v along n, t1, t2 (B minus A; static ends have v = 0) / (g_ref h)
 *   3    penetration max(-phi, 0) / (g_ref h^2)
 *   4-6  the previous-step impulses the plain warm start applies / s
 *   7-8  inverse masses of A and B (0 for a static end or a plane)
 *   9-10 degrees of A and B in G^t / 8 (0 for a static end)
 *   11   min over the dynamic ends of the BFS distance in G^t to the nearest
 *        body of O, capped at 8, / 8
 * The network's three outputs y are impulses / s; features 4-6 feed them
 * directly, so the layers learn a correction to the method's own warm start.
 * The warm start is s y with the normal impulse made non-negative and each
 * friction impulse clamped to +-mu times it.  Inference uses BF16 operands with FP32 accumulation on the
 * tensor cores.  Training reads a log of (features, impulses / s) pairs that
 * steps append, minimises the mean squared error with Adam, and runs in the
 * library's own forward and backward kernels (BF16 operands, FP32 sums, FP32
 * master parameters).
 *
 * Parameter vector (OVL_MLP_N_PARAMS floats): W1 [12][64] (input-major), b1
 * [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3]; y = x[4:7] + W3^T
 * relu(W2^T relu(W1^T x + b1) + b2) + b3.
 * ------------------------------------------------------------------------ */
#define OVL_MLP_N_PARAMS 5187
#define OVL_N_FEATURES 12

/* OVL_WS_PREVIOUS, OVL_WS_MLP or OVL_WS_MLP_NEW for the following steps.
 * The MLP modes need parameters (ovl_mlp_set_params). */
ovl_status ovl_set_warmstart_mode(ovl_ctx *ctx, int32_t mode);

/* Per (worker, constraint) pair of the last step, in ovl_read_pairs order
 * (host outputs, n_pairs rows; any may be NULL): the features [12] (zero for
 * joints), the scale s (0 for joints), 1 if previous impulses existed, and
 * the warm-start impulses [3] the solve started from.  OVL_ERR_ARG if the
 * last step computed no features (plain mode without OVL_FLAG_FEATURES or
 * logging). */
ovl_status ovl_read_features(ovl_ctx *ctx, float *feat12, float *scale, int32_t *found,
                             float *lambda0_3);

/* Sets / reads the network's parameters (host arrays of n =
 * OVL_MLP_N_PARAMS floats).  Setting them also resets Adam's moments and
 * step count. */
ovl_status ovl_mlp_set_params(ovl_ctx *ctx, const float *theta, int32_t n);
ovl_status ovl_mlp_get_params(ovl_ctx *ctx, float *theta, int32_t n);

/* The network's raw outputs y [n][3] for host features [n][12] (the same
 * kernel the step uses). */
ovl_status ovl_mlp_forward(ovl_ctx *ctx, int64_t n, const float *feat12, float *y3);

/* The training log: rows of (features [12], target impulses / s [3]) in
 * device memory.  reserve: allocates room for capacity rows (0 frees) and
 * empties it.  enable: while on, every step appends its contact pairs with
 * the impulses its solve ended with (rows beyond the capacity are dropped).
 * append / read: host rows in and out, e.g. for data made elsewhere. */
ovl_status ovl_log_reserve(ovl_ctx *ctx, int64_t capacity);
ovl_status ovl_log_enable(ovl_ctx *ctx, int32_t on);
ovl_status ovl_log_size(ovl_ctx *ctx, int64_t *n);
ovl_status ovl_log_append(ovl_ctx *ctx, int64_t n, const float *feat12, const float *target3);
ovl_status ovl_log_read(ovl_ctx *ctx, int64_t first, int64_t n, float *feat12, float *target3);

typedef struct ovl_train_desc {
    int64_t first, count;  /* log rows [first, first + count) */
    int32_t batch;         /* samples per Adam step, 1 .. 1048576 */
    int32_t steps;         /* Adam steps */
    int32_t sampling;      /* 0: consecutive batches cycling through the rows; 1: rows drawn
                              uniformly with replacement (SplitMix64 of seed and sample index) */
    float lr, beta1, beta2, eps;   /* Adam (defaults 1e-3, 0.9, 0.999, 1e-8) */
    uint64_t seed;
} ovl_train_desc;

/* Runs desc->steps Adam steps on the mean squared error of the scaled
 * impulses; loss_per_step (host, may be NULL) receives the loss of each
 * step's batch before its update. */
ovl_status ovl_mlp_train(ovl_ctx *ctx, const ovl_train_desc *desc, float *loss_per_step);

/* Gradient [OVL_MLP_N_PARAMS] and loss of the mean squared error over the
 * log rows [first, first + count) at the current parameters (no update);
 * count <= 1048576. */
ovl_status ovl_mlp_grad(ovl_ctx *ctx, int64_t first, int64_t count, float *grad, double *loss);

/* Mean squared error over the log rows [first, first + count). */
ovl_status ovl_mlp_loss(ovl_ctx *ctx, int64_t first, int64_t count, double *loss);

/* ------------------------------------------------------------------------
 * Geodesic distances without allocation
 *
 * No counterpart in the paper.  Computes the same D(o,i) as the geodesic
 * phase of ovl_step (the distance, in edges of the constraint graph, from
 * overlap body o to the nearest body that only worker i simulates, cut at
 * depth beta), for one scene whose graph, masks and entries the caller
 * already holds on the device.  It exists for callers that must not allocate
 * device memory: fixed-rate control loops, where cudaFree synchronises the
 * whole device and stalls every other stream for an unbounded time; and
 * programs that give all device memory to their own pool at start-up, where
 * a library's cudaMalloc would fail or break the pool's accounting.  The
 * function calls neither cudaMalloc nor cudaFree nor any
 * allocating library routine: its search bitmap, frontier queue and level
 * counters live in one statically sized __device__ array of the library
 * (about 16.5 MiB) that every GPU which loads the library holds until the
 * process exits.  Its device address is looked up in the current device's
 * context on every call, so a device reset needs no special handling.
 *
 * Limits: n_bodies * n_workers <= OVL_GEO_STATIC_MAX_PAIRS and
 * beta <= OVL_GEO_STATIC_MAX_BETA; larger problems are rejected with
 * OVL_ERR_CAPACITY before anything runs (use ovl_step for them).
 *
 * Arguments (all arrays are DEVICE pointers owned by the caller):
 *  n_bodies            bodies of the scene; n_workers in [1, 64]; beta >= 0
 *  row_ptr [n_bodies+1], col [n_adj]: G^t as CSR (body indices < n_bodies)
 *  mask [n_bodies]     W_b, bit i set when worker i simulates body b; bits at
 *                      or above n_workers are ignored
 *  entry_ptr [n_bodies+1], n_entries: the entries of body b are
 *                      entry_ptr[b] .. entry_ptr[b+1]-1, one per bit of
 *                      mask[b] in ascending worker order (ovl_read_entries)
 *  D [n_entries]       out: D(o,i) for bodies with two or more workers, 255
 *                      where worker i was not met within beta and for every
 *                      entry of a body with one worker
 *  cuda_stream         cudaStream_t to enqueue on (NULL: the legacy stream);
 *                      the call returns once the work is enqueued
 *  err, err_cap        optional buffer for a NUL-terminated message on error
 * Indices out of range (col, entry_ptr) are skipped, never dereferenced.
 *
 * Concurrency: the scratch array is shared by every call on a device, so
 * two calls whose work can overlap on the device (other streams, other
 * threads, or other processes sharing a context) race and give wrong D.
 * Serialise them, e.g. on one stream.  The array keeps the last call's
 * contents; each call clears the parts it reads before it uses them.  The
 * first call on each device (and the first after a device reset) may load
 * the library's module while it looks up the address
 * (cudaGetSymbolAddress); make that call before any stream capture begins. */
#define OVL_GEO_STATIC_MAX_PAIRS 4194304
#define OVL_GEO_STATIC_MAX_BETA 254
ovl_status ovl_geodesics_static(int32_t n_bodies, int32_t n_workers, int32_t beta,
                                const int32_t *row_ptr, const int32_t *col, int32_t n_adj,
                                const uint64_t *mask, const int32_t *entry_ptr,
                                int32_t n_entries, uint8_t *D, void *cuda_stream, char *err,
                                int32_t err_cap);

#ifdef __cplusplus
}
#endif

#endif /* OVL_H */
