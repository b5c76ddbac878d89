// ctx.cuh -- the library context (ovl_ctx) and the host helpers the
// translation units of the C ABI share.
#pragma once

#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

using namespace ovl;

struct ovl_ctx {
    ovl_params P{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int smem_optin = 0;
    int num_sms = 0;
    int smem_per_sm = 0;
    int nb_max = 0;          // most bodies in one worker (last membership phase)
    int last_cluster = 1, last_threads = 512, last_unroll = 1;
    bool last_plan_per_worker = false;   // the last solve used h_class_C (else last_cluster for all)
    long long last_ctas = 0, last_ctas_masses = 0;   // CTAs of the last solve, those with masses in shared memory
    // a tuned solve launch: uniform (cluster > 0) or per-worker plan (shape = 1 + its index)
    struct TuneCfg { int cluster, threads, unroll; float ms; int shape; };
    std::map<std::string, TuneCfg> tuned;   // autotuner results by problem-size bucket
    std::string err;

    // scene (host copies)
    bool has_scene = false;
    bool has_boxes = false;          // some body has positive half extents
    std::vector<float> h_half;       // [n][3] half extents (zeros: a sphere)
    HostScene hs;
    int n = 0, np = 0, nj = 0, ns = 0, n_parts = 0, beta_max = 0;
    std::vector<float> h_radius, h_im;
    std::vector<int> h_body_base, h_plane_ptr, h_part_scene;
    float cs = 1.f;
    uint32_t tsize = 0;
    long long vb_bits = 0;

    // scene (device)
    DBuf<float4> st, st_alt;
    DBuf<float> radius, im, scene_mu, scene_dt;
    DBuf<int> sob, scene_flags, n_sets, part_base, body_base, scene_beta, scene_gamma, joint_scene, part_scene;
    DBuf<float4> planes;
    DBuf<int> plane_ptr, plane_list;
    DBuf<int2> jab;
    DBuf<float4> janc;
    DBuf<long long> vb_base;
    DBuf<uint64_t> mask;
    DBuf<float4> half, iib;   // boxes: half extents; body-frame inverse inertia diagonal (1/I_x, 1/I_y, 1/I_z)

    // step buffers
    DBuf<int> status;
    DBuf<int4> cell;
    DBuf<int> bucket_count, bucket_start, cursor, items, nb_list, nb_count, ccount, cstart;
    DBuf<long long> nb_off;    // per-body neighbour capacity offsets (set at scene upload)
    long long nb_total = 0;
    DBuf<int2> c_ab;
    DBuf<float4> c_n, c_t1;
    DBuf<float4> c_p;          // contact point, manifold index in w (contexts with boxes)
    DBuf<int> deg, tptr, cursor2, tcol, ucount, row_ptr, col;
    DBuf<int> entry_count, entry_ptr, entry_body, entry_part, entry_slot, part_list, part_count,
        part_bstart;
    DBuf<uint32_t> sk, sv, sk2, sv2;
    DBuf<int> cons_count, cons_start, pair_cons, pair_part, ps_cons, ps_part, part_pcount,
        part_pstart, p_colour, part_ncol, part_rounds, col_off, pair_of_row;
    DBuf<uint64_t> p_key;
    DBuf<int2> p_slot;
    DBuf<float4> p_lam0;
    DBuf<unsigned long long> colour_scratch;
    DBuf<int4> worklist, worklist2;
    DBuf<unsigned long long> wprio, wprio2;
    DBuf<float4> r0, r1, r2, r3, rlam, lam_out;
    DBuf<int> rpair;
    DBuf<int> ws_pstart;
    DBuf<uint64_t> ws_key;
    DBuf<float4> ws_lam;
    int64_t ws_n = 0;
    DBuf<float4> copies, solve_scratch;
    DBuf<int> part_iters;
    DBuf<double> part_res_sq;
    DBuf<uint32_t> visited, queue;
    DBuf<int> qctl;
    DBuf<uint8_t> D;
    DBuf<float> weight;
    DBuf<float> stage13;   // staging for host <-> device state transfers
    DBuf<int> scan_tmp, sort_hist, sort_tmp;
    HBuf<int> h_i32;
    HBuf<int2> h_ab;
    HBuf<int> h_rp, h_col;
    HBuf<uint64_t> h_mask;
    DBuf<int> lb_flag, lb_pos;
    DBuf<int> ball_root, ball_size, ball_start, ball_vtx, ball_list;   // Algorithm 6's gamma-balls, found ahead
    HBuf<int> h_ball_start, h_ball_vtx;
    DBuf<int2> lb_pairs;
    DBuf<uint32_t> worker_order, wk, wk2, wv2;   // workers longest first (launch order)
    DBuf<uint32_t> class_order, colour_order;    // solve / colouring: workers grouped by CTAs per worker
    std::vector<int> h_pb, h_pp;                 // part_bstart, part_pstart of this step on the host
    std::vector<int> h_class_C;                  // CTAs per worker of the last per-worker plan
    DBuf<int> solve_C, solve_M, col_off2, pair_of_row2;   // solve: CTAs per worker, masses in shared memory, rows by owner CTA
    DBuf<uint8_t> row_owner;                     // owner CTA of every row (scratch of the grouping)
    DBuf<uint8_t> row_full;                      // rows with a box end (contexts with boxes)
    DBuf<float4> rfull;                          // their records, FULL_ROW_WORDS float4 per row
    cudaStream_t aux[6] = {};                    // per-class launches, priorities falling with the index
    cudaStream_t geo_stream = nullptr;           // the geodesic weights, beside colouring and solve
    cudaEvent_t geo_fork = nullptr, geo_join = nullptr;
    cudaEvent_t fork = nullptr, join[6] = {};
    cudaGraphExec_t geo_exec = nullptr;          // the geodesic phase, captured
    std::vector<const void *> geo_key;           // its arguments when captured
    long long geo_kernels = 0;
    int lb_threads = 1;            // host threads of the load balance (scenes run in parallel)
    std::vector<BallWorkspace> lb_ws;
    DBuf<int> lb_loads;
    HBuf<int> h_loads;
    DBuf<int> lb_deg;          // contacts per body (contact load)
    DBuf<double> jerr;         // joint error: sum, max
    HBuf<int> h_deg;

    // last step
    int64_t step_index = 0;
    int nc = 0, nadj = 0, ne = 0, npairs = 0;
    bool have_step = false;
    cudaEvent_t ev[16] = {};
    float phase_ms[12] = {};
    long long last_launches = 0;
    long long lb_candidates = 0;
    double lb_host_ms = 0.0;

    // learned warm start
    int ws_mode = OVL_WS_PREVIOUS;
    bool feat_valid = false;          // the last step computed features
    DBuf<float4> feat;                // [np][4]
    DBuf<int> is_contact, contact_pos;
    DBuf<uint8_t> depth;
    bool mlp_ready = false;           // parameters were set
    DBuf<float> mlp_theta, mlp_m, mlp_v, mlp_grad, mlp_loss;
    DBuf<uint32_t> mlp_packed;
    long long adam_t = 0;
    DBuf<float> log_feat, log_targ;
    long long log_cap = 0, log_n = 0;
    bool log_on = false;
    DBuf<float> train_act, train_sample_loss, train_partials, train_loss_hist, infer_y;
    DBuf<float4> infer_feat;
    DBuf<double> loss_acc;
    DBuf<float> train_c12;            // Adam bias corrections per step of a training call
    DBuf<long long> train_step;       // step counter of a training call (graph replay)
};

namespace ovl {

inline ovl_status fail(ovl_ctx *c, ovl_status code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

template <class F>
ovl_status guarded(ovl_ctx *c, F &&f) {
    if (!c) return OVL_ERR_ARG;
    try {
        return f();
    } catch (const CudaError &e) {
        return fail(c, OVL_ERR_CUDA, std::string(e.what) + ": " + cudaGetErrorString(e.err));
    } catch (const std::bad_alloc &) {
        return fail(c, OVL_ERR_CUDA, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(c, OVL_ERR_ARG, e.what());
    }
}

inline int read_i32(ovl_ctx *c, const int *dptr) {
    c->h_i32.ensure(1);
    CK(cudaMemcpyAsync(c->h_i32.p, dptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return c->h_i32.p[0];
}

template <class T>
void upload(DBuf<T> &buf, const T *src, size_t n, cudaStream_t s) {
    buf.ensure(n ? n : 1);
    if (n) CK(cudaMemcpyAsync(buf.p, src, sizeof(T) * n, cudaMemcpyHostToDevice, s));
}

template <class T>
void download(T *dst, const T *src, size_t n, cudaStream_t s) {
    if (n) CK(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
}

// the step's device status word as an ovl_status (and the message)
ovl_status check_device_status(ovl_ctx *c);

// learned warm start (mlp.cu): features and the network's proposal before
// the rows are built; the log after the solve; buffers freed with the context
void phase_warmstart(ovl_ctx *c, float dt_override);
void phase_log(ovl_ctx *c);
void release_mlp(ovl_ctx *c);

}  // namespace ovl
