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
    int *nb_list;          // [n][OVL_MAX_NEIGH]
    int *nb_count;         // [n]
    int *contact_count;    // [n+1]
    int *contact_start;    // [n+1]
    int2 *c_ab;
    float4 *c_n;
    float4 *c_t1;
    int *status;
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
void launch_lb_flags(const int2 *c_ab, int nc, const float *im, int n, const uint64_t *mask,
                     int disjoint_only, int *flag, cudaStream_t s);
void launch_lb_compact(const int2 *c_ab, int nc, const int *flag, const int *pos, int2 *out,
                       cudaStream_t s);
void launch_adj_compact(const int *tptr, const int *tcol, int n, const int *row_ptr, int *col,
                        cudaStream_t s);

// ---- membership, pairs, warm start, colouring, rows (k_member.cu) ----------
struct MemberArgs {
    int n, nc, nj, n_parts;
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

struct ColourArgs {
    int n_parts;
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
    int4 *worklist, *worklist2;                 // [np] each: uncoloured constraints per round
    unsigned long long *wprio, *wprio2;         // [np] each: their priorities
    int smem_slots;            // slots that fit in shared memory
    int *status;
};
void launch_colour(const ColourArgs &a, int cluster, cudaStream_t s);

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
    float4 *r0, *r1, *r2, *r3;
    int *rpair;                // [np] pair index of every row (canonical order)
    float4 *rlam;
    int *status;
};
void launch_rows(const RowArgs &a, cudaStream_t s);

// ---- PGS solve + integration (k_solve.cu) ----------------------------------
struct SolveArgs {
    int n_parts;
    const int *part_bstart;
    const int *part_list;
    const int *entry_body;
    const int *part_ncol;
    const int *col_off;
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
};
void launch_solve(const SolveArgs &a, int threads, int cluster, int unroll, cudaStream_t s);
int solve_ctas_per_sm(int unroll);
int solve_smem_bytes(int slots);

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
    int *status;
};
void launch_blend(const BlendArgs &a, cudaStream_t s);

// state conversion [n][13] <-> 64-byte records
void launch_pack_state(const float *in13, const float *radius, const float *im, int n, float4 *st,
                       cudaStream_t s);
void launch_unpack_state(const float4 *st, int n, float *out13, cudaStream_t s);

}  // namespace ovl
