// kernels.cuh -- argument blocks and host launchers of the step's kernels.
#pragma once

#include "common.cuh"

namespace ovl {

int grid1d(size_t n, int threads);

// ---- contacts and constraint graph (k_contacts.cu) -------------------------
struct ContactArgs {
    const float4 *st;      // body state, 4 float4 per body
    const float *im;       // inverse mass
    int n;
    const int *sob;
    const int *scene_flags;
    float inv_cs;
    uint32_t tmask;        // hash table size - 1
    int4 *cell;            // per body (ix, iy, iz, hash)
    int *bucket_count;     // [T]
    int *bucket_start;     // [T+1]
    int *cursor;           // [T]
    int *items;            // [n]
    const float4 *planes;
    const int *plane_ptr;  // [n_scenes+1]
    const int *plane_list; // plane indices grouped by scene, ascending
    float margin;
    int *nb_list;          // per body a range of nb_off[b + 1] - nb_off[b] entries
    const long long *nb_off; // [n+1] neighbour-list offsets (per-body capacity from the radii)
    int *nb_count;         // [n]
    int *contact_count;    // [n+1]
    int *contact_start;    // [n+1]
    int2 *c_ab;
    float4 *c_n;
    float4 *c_t1;
    int *status;
    const float4 *half;    // [n] box half extents (w unused), or NULL: no box in the context
    float4 *c_p;           // [nc] contact point and, as int bits in w, the manifold index (box contexts)
};
void launch_cells(const ContactArgs &a, cudaStream_t s);
void launch_bucket_fill(const ContactArgs &a, cudaStream_t s);
void launch_find_pairs(const ContactArgs &a, cudaStream_t s);
void launch_write_contacts(const ContactArgs &a, cudaStream_t s);
void launch_edge_degree(const int2 *c_ab, int nc, const int2 *jab, int nj, const float *im, int n,
                        int *deg, cudaStream_t s);
void launch_edge_fill(const int2 *c_ab, int nc, const int2 *jab, int nj, const float *im, int n,
                      const int *tptr, int *cursor, int *tcol, cudaStream_t s);
void launch_adj_unique(const int *tptr, int n, int *tcol, int *ucount, cudaStream_t s);
// loads [P] := |P_w| of every worker from the masks
// number of contacts each body is an end of (planes and static ends included)
void launch_contact_degree(const int2 *c_ab, int nc, int n, int *deg, const float4 *c_p, cudaStream_t s);
// load of every worker: sum over its active bodies of 1 (+ deg[b] when deg != NULL)
void launch_worker_loads(const uint64_t *mask, const int *sob, const int *part_base, const int *deg, int n, int P,
                         int *loads, cudaStream_t s);
void launch_lb_flags(const int2 *c_ab, int nc, const float *im, int n, const uint64_t *mask,
                     int disjoint_only, int *flag, const float4 *c_p, cudaStream_t s);
void launch_lb_compact(const int2 *c_ab, int nc, const int *flag, const int *pos, int2 *out,
                       cudaStream_t s);
// Algorithm 6's gamma-balls, found ahead of the host pass: root[v] = 1 and v
// in list[0..*count) for the ends of the m candidate contacts whose masks
// are disjoint (root, count zeroed by the caller; list holds up to 2m);
// size[v] the ball's vertex count (0: not a root or too large; zeroed by the
// caller); vtx at start[v] (the exclusive scan of size) the vertices
void launch_ball_roots(const int2 *ab, int m, const uint64_t *mask, int *root, int *list, int *count,
                       cudaStream_t s);
void launch_balls(bool fill, int max_roots, const int *list, const int *count, const int *row_ptr, const int *col,
                  const int *sob, const int *scene_gamma, int *size, const int *start, int *vtx, cudaStream_t s);
void launch_adj_compact(const int *tptr, const int *tcol, int n, const int *row_ptr, int *col,
                        cudaStream_t s);

// ---- membership, pairs, warm start, colouring, rows (k_member.cu) ----------
struct MemberArgs {
    int n, nc, nj, n_parts;
    const float4 *c_p;         // contexts with boxes: manifold index of every contact (w), else NULL
    const float *im;
    const int *sob;
    const int *n_sets;       // per scene
    const int *part_base;    // per scene (+1)
    const int *joint_scene;
    const uint64_t *mask;
    const int2 *c_ab;
    const int2 *jab;
    // entries
    int *entry_count;        // [n+1]
    int *entry_ptr;          // [n+1]
    int *entry_body;         // [ne]
    int *entry_part;         // [ne]
    int *entry_slot;         // [ne]
    int *part_list;          // [ne] entries grouped by worker, bodies ascending
    int *part_bstart;        // [P+1]
    // pairs
    int *cons_count;         // [nc+nj+1]
    int *cons_start;         // [nc+nj+1]
    int *pair_cons;          // [np] canonical (constraint-major)
    int *pair_part;          // [np]
    int *ps_cons;            // [np] grouped by worker, canonical inside
    int *ps_part;            // [np]
    int *part_pstart;        // [P+1]
    uint64_t *p_key;         // [np]
    int2 *p_slot;            // [np] worker-local slots of the two ends (-1 static)
    float4 *p_lam0;          // [np] warm-start impulses
    int *status;
};
void launch_entry_count(const MemberArgs &a, cudaStream_t s);
void launch_entry_fill(const MemberArgs &a, cudaStream_t s);
void launch_entry_slot(const MemberArgs &a, int ne, cudaStream_t s);
void launch_cons_count(const MemberArgs &a, cudaStream_t s);
void launch_pair_fill(const MemberArgs &a, cudaStream_t s);
void launch_pair_gather(const MemberArgs &a, const uint32_t *order, int np, cudaStream_t s);

struct WarmArgs {
    const int *ws_pstart;      // [P+1] previous step's (worker) ranges
    const uint64_t *ws_key;    // sorted keys per worker
    const float4 *ws_lam;
    float factor;
};
void launch_pair_setup(const MemberArgs &a, const WarmArgs &w, int np, cudaStream_t s);
// Rows of every colour regrouped by the CTA that owns them in the solve:
// worker p's bodies are split into solve_C[p] contiguous slot ranges of
// ceil(nb / C) slots, one per CTA, and a row belongs to the CTA holding its
// first dynamic body.  off_in: [P][2*OVL_MAX_COLOURS+1] (colour, kind)
// offsets of pair_of_row; off_out: [P][OWNER_NB] offsets of (colour, owner
// rank, kind) buckets, ranks 0..7, contacts before joints, then the end.
#define OWNER_RANKS 8
#define OWNER_NB (OVL_MAX_COLOURS * OWNER_RANKS * 2 + 1)
void launch_row_owner(int P, const int *part_bstart, const int *part_ncol, const int *solve_C,
                      const int *off_in, const int *pair_of_row, const int2 *p_slot,
                      uint8_t *owner_of_row, int *pair_of_row_out, int *off_out, cudaStream_t s);
// keys[p] = 2^24 - 1 - min(pairs of worker p, 2^24 - 1), vals[p] = p: an
// ascending stable sort of the keys lists the workers longest first
void launch_worker_cost_keys(const int *part_pstart, int P, uint32_t *keys, uint32_t *vals,
                             cudaStream_t s);

struct ColourArgs {
    int n_parts;
    const uint32_t *order;     // [P] worker of each CTA group, longest first (NULL: identity)
    const int *part_list;      // [ne] entries grouped by worker, bodies ascending
    const int *entry_body;     // [ne]
    const int *part_bstart;
    const int *part_pstart;
    const uint64_t *p_key;
    const int2 *p_slot;
    int *p_colour;             // [np]
    int *part_ncol;            // [P]
    int *part_rounds;          // [P] colouring rounds taken
    int *col_off;              // [P][2*OVL_MAX_COLOURS+1] absolute row offsets per (colour, kind)
    int *pair_of_row;          // [np]
    unsigned long long *scratch;  // 2 per entry, for workers too large for shared memory
    unsigned long long *hi_mask;  // [ne] colours 64-127 taken at every worker slot
    int4 *worklist, *worklist2;                 // [np] each: uncoloured constraints per round
    unsigned long long *wprio, *wprio2;         // [np] each: their priorities
    int smem_slots;            // slots that fit in shared memory
    int *status;
};
void launch_colour(const ColourArgs &a, int cluster, cudaStream_t s);
int colour_static_smem();

struct RowArgs {
    int n, nc, np;
    const int *pair_of_row;
    const int *ps_cons;
    const int *ps_part;
    const int2 *p_slot;
    const float4 *p_lam0;
    const int2 *c_ab;
    const float4 *c_n;
    const float4 *c_t1;
    const int2 *jab;
    const float4 *janc;        // 2 per joint (anchor a, anchor b)
    const int *joint_scene;
    const float4 *st;
    const int *sob;
    const int *part_scene;
    const float *scene_dt;
    const float *scene_mu;
    float dt_override;
    float erp, slop;
    float4 *r0, *r1, *r2, *r3;   // r2: joints only
    const int *part_bstart;      // [P+1] worker slot ranges
    const int *solve_C;          // [P] CTAs per worker in the solve plan (slot codes)
    const int *solve_M;          // [P] 1: the worker's launch keeps the masses in shared memory (or NULL)
    int *rpair;                // [np] pair index of every row (canonical order)
    float4 *rlam;
    int *status;
    // contexts with boxes (else NULL): contact points, half extents, body-frame
    // inverse inertia diagonals; out: the full-row flag and record of every row
    const float4 *c_p, *half, *iib;
    uint8_t *row_full;
    float4 *rfull;
};
void launch_rows(const RowArgs &a, cudaStream_t s);

// A constraint with a box end (a contact touching a box, or a ball joint with
// a box end) is a "full" row: its lever arms reach the contact point (or the
// pivots) and a box's angular response is its world inverse inertia
// R diag(1/I) R^T.  Per constraint FULL_ROW_WORDS float4, for its three
// directions d_i (contact: n, t1, t2 = n x t1; joint: the world axes):
//   [i]      (d_i, target_i)
//   [3 + i]  (r_A x d_i, k_i)                k_i = 1 / (J_i M^-1 J_i^T)
//   [6 + i]  (I_A^-1 (r_A x d_i), 0)
//   [9 + i]  (r_B x d_i, 0)
//   [12 + i] (I_B^-1 (r_B x d_i), 0)
//   [15]     (1/m_A, 1/m_B, 0, 0)            (0 for a static end or one not in the worker)
// The row's velocity is d_i.(v_B - v_A) + (r_B x d_i).w_B - (r_A x d_i).w_A.
#define FULL_ROW_WORDS 16

// ---- PGS solve + integration (k_solve.cu) ----------------------------------
struct SolveArgs {
    int n_parts;
    const uint32_t *order;     // [P] worker of each CTA group, longest first (NULL: identity)
    const int *part_bstart;
    const int *part_list;
    const int *entry_body;
    const int *part_ncol;
    const int *col_off;        // [P][OWNER_NB] (colour, owner rank, kind) row offsets
    const int *part_scene;
    const float *scene_dt;
    float dt_override;
    float3 gravity;
    const float4 *st;
    const float *scene_mu;
    const float4 *r0, *r1, *r2, *r3;
    const int *rpair;
    float4 *rlam;
    int n_entries;
    float4 *lam_out;           // [np] canonical pair order
    float4 *copies;            // [ne][4]
    float4 *scratch;           // [ne] float4 + [ne] float2: velocities of workers too large for shared memory
    int iters;
    int smem_slots;
    int flags;                 // OVL_FLAG_*
    float res_tol;
    int res_check_every;
    int *part_iters;           // [P]
    double *part_res_sq;       // [P]
    int *status;
    const uint8_t *row_full;   // contexts with boxes: rows read from rfull (FULL_ROW_WORDS each), else NULL
    const float4 *rfull;
};
// masses: the shared-memory slots hold the inverse masses and inertias (32 B
// per slot; contact rows read as two records); else 24 B per slot
void launch_solve(const SolveArgs &a, int threads, int cluster, int unroll, bool masses, cudaStream_t s);
int solve_ctas_per_sm(int unroll);
int solve_slot_bytes(bool masses);              // bytes of one shared-memory body slot
int solve_smem_bytes(int slots, bool masses);   // a CTA's slots plus its zero slot

// ---- geodesics, weights, blend (k_blend.cu) --------------------------------
struct GeoArgs {
    int n;
    const uint64_t *mask;
    const int *sob;
    const int *scene_beta;
    const int *body_base;      // per scene
    const long long *vb_base;  // per scene: first bit of its (worker, body) bitmap
    const int *row_ptr;
    const int *col;
    const int *entry_ptr;
    uint32_t *visited;         // bitmap
    uint32_t *queue;           // (body << 6 | worker)
    int *qctl;                 // [0] = tail, [1 + L] = start of level L
    uint8_t *D;                // per entry
};
void launch_geo_sources(const GeoArgs &a, cudaStream_t s);
void launch_geo_level(const GeoArgs &a, int level, cudaStream_t s);

struct BlendArgs {
    int n;
    const int *entry_ptr;
    const uint8_t *D;
    const float4 *copies;
    const float4 *st_in;
    float4 *st_out;
    float *weight;             // per entry (recorded for read-back)
    const int *sob;
    const float *scene_dt;
    float dt_override;
    int uniform;               // 1: weights 1 / |W_b| instead of Eq 15-16
    int *status;
};
void launch_blend(const BlendArgs &a, cudaStream_t s);
// sum and max of the pivot gaps of nj ball joints over a [n] x 4 float4 state
// (out[0] = sum, out[1] = max); one CTA, fixed reduction order
void launch_joint_error(const int2 *jab, const float4 *janc, const float4 *st, int nj, double *out,
                        cudaStream_t s);

// state conversion [n][13] <-> 64-byte records
void launch_pack_state(const float *in13, const float *radius, const float *im, int n, float4 *st,
                       cudaStream_t s);
void launch_unpack_state(const float4 *st, int n, float *out13, cudaStream_t s);

// ---- learned warm start (k_mlp.cu) ------------------------------------------
// Per pair, 16 floats: the 12 features, then previous-impulses flag, scale s,
// friction coefficient, contact flag (1 for contacts, 0 for joints).
#define MLP_DEPTH_CAP 8
#define MLP_N_PARAMS 5187
#define MLP_PK_WORDS 3216      // BF16 tensor-core operands + FP32 biases
#define MLP_ACT_STRIDE 276     // x 16, h1 64, h2 64, dz1 64, dz2 64, dy 4
struct FeatArgs {
    int np, nc, n;
    const int *ps_cons, *ps_part, *part_scene;
    const int2 *c_ab;
    const float4 *c_n, *c_t1;
    const float4 *st;
    const int *row_ptr;
    const uint8_t *depth;
    const float *scene_dt, *scene_mu;
    float dt_override;
    float g_ref;
    const uint64_t *p_key;
    WarmArgs ws;
    float4 *feat;              // [np][4]
    int *is_contact;           // [np]
};
void launch_depth(const uint64_t *mask, const int *row_ptr, const int *col, int n, uint8_t *depth,
                  cudaStream_t s);
void launch_features(const FeatArgs &a, cudaStream_t s);
void launch_mlp_pack(const float *theta, uint32_t *packed, cudaStream_t s);
// mode 0: raw outputs to y3 [n][3]; 1: warm start of every contact into lam0;
// 2: warm start of the contacts without previous impulses into lam0.  On the
// tensor cores (tcgen05); a wait on them that gives up sets *status to
// DEV_ERR_TIMEOUT.
void launch_mlp_infer(const uint32_t *packed, const float4 *feat, int n, int mode, float4 *lam0,
                      float *y3, int grid_limit, int *status, cudaStream_t s);
void launch_log_append(const float4 *feat, const float4 *lam, const int *pos, int np,
                       float *log_feat, float *log_targ, long long base, long long cap,
                       cudaStream_t s);

struct TrainArgs {
    const float *log_feat, *log_targ;   // [rows][12], [rows][3]
    long long first, count;             // rows sampled from [first, first + count)
    int batch;
    int sampling;                       // 0 contiguous, 1 uniform with replacement
    unsigned long long seed;
    long long step;                     // Adam step within the call (sampling)
    const long long *step_dev;          // if set: the step counter in device memory (graph replay)
    int backward;                       // 0: loss only
    const float *theta;                 // FP32 master parameters
    float *act;                         // [batch][MLP_ACT_STRIDE]
    float *sample_loss;                 // [batch]
    float *partials;                    // [blocks][MLP_N_PARAMS + 1]
    int *status;                        // set to DEV_ERR_TIMEOUT if a tensor-core wait gives up
};
void launch_train_fwd(const TrainArgs &a, cudaStream_t s);
int train_wgrad_blocks(int batch);
// Function attributes of the network's kernels on `device`: once per context,
// before any of their launches (outside graph capture).
void mlp_kernels_setup(int device);
void launch_train_wgrad(const TrainArgs &a, cudaStream_t s);
// sums the partials in block order; grad_out (optional) gets the gradient and
// loss_out[0] the mean loss; with adam != 0 also updates theta, m, v
void launch_train_reduce(const float *partials, int blocks, int batch, float *grad_out,
                         float *loss_out, int adam, float *theta, float *m, float *v, float lr,
                         float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s);
// the same with the step taken from step_dev: loss to loss_hist[step], bias
// corrections from c12[2 step], c12[2 step + 1]; then step_dev += 1
void launch_train_reduce_dev(const float *partials, int blocks, int batch, float *loss_hist,
                             float *theta, float *m, float *v, float lr, float beta1, float beta2,
                             float eps, const float *c12, long long *step_dev, cudaStream_t s);
void launch_loss_sum(const float *sample_loss, int n, double *acc, cudaStream_t s);

}  // namespace ovl
