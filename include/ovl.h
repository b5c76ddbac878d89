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
#define OVL_ERR_CAPACITY (-3)   /* a fixed limit was exceeded (colours > 64, neighbours > 32, ...) */
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
} ovl_params;

#define OVL_FLAG_RESIDUAL 1  /* compute the complementarity residual of every row after the sweeps */
#define OVL_FLAG_TIMING 2    /* record per-phase times with CUDA events (ovl_read_stats) */
#define OVL_FLAG_AUTOTUNE 4  /* time the solver's launch shapes on the first step of every problem-size
                                bucket and keep the fastest (results are bit-identical across shapes) */

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
    float phase_ms[12];        /* per-phase device times (OVL_FLAG_TIMING); see ovl_phase_name */
    int64_t n_launches;        /* CUDA kernels the library launched during the last step */
    int32_t solve_cluster;     /* CTAs per worker of the last solve */
    int32_t solve_threads;     /* threads per CTA of the last solve */
    int32_t solve_rows_per_thread; /* rows a thread takes at once in a colour (colour block) */
    int32_t colour_rounds_max; /* most colouring rounds any worker needed */
    int64_t lb_candidates;     /* contacts handed to the host load balance in the last step */
    double lb_host_ms;         /* host time of the load balance in the last step (copies included) */
} ovl_stats;

/* Fills *p with the defaults listed in ovl_params. */
ovl_status ovl_default_params(ovl_params *p);

/* Creates a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * to run on, or NULL for a stream the context owns.  *out receives the
 * context; destroy it with ovl_destroy. */
ovl_status ovl_create(ovl_ctx **out, const ovl_params *p, void *cuda_stream);
ovl_status ovl_destroy(ovl_ctx *ctx);
const char *ovl_last_error(const ovl_ctx *ctx);
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

/* Per worker: sweeps run, residual sum of squares, rows, colours. */
ovl_status ovl_read_worker_stats(ovl_ctx *ctx, int32_t *iters, double *res_sq, int64_t *rows,
                                 int32_t *colours);

/* ------------------------------------------------------------------------
 * Geodesic distances without allocation
 *
 * No counterpart in the paper.  Computes the same D(o,i) as the geodesic
 * phase of ovl_step (Eq 16, Algorithm 5: breadth-first search over the
 * constraint graph G^t from the bodies that only worker i simulates, cut at
 * depth beta), for one scene whose graph, masks and entries the caller
 * already holds on the device.  It exists for callers that must not allocate
 * device memory: fixed-rate control loops, where cudaFree synchronises the
 * whole device and stalls every other stream for an unbounded time; and
 * programs that give all device memory to their own pool at start-up, where
 * a library's cudaMalloc would fail or break the pool's accounting.  The
 * function calls neither cudaMalloc nor cudaFree nor any
 * allocating library routine: its search bitmap, frontier queue and level
 * counters live in one statically sized __device__ array of the library
 * (about 16.5 MiB), whose device address is looked up once per device.
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
 * Serialise them, e.g. on one stream.  The first call on each device looks
 * up the scratch address (cudaGetSymbolAddress, which may load the module);
 * make that first call before any stream capture begins. */
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
