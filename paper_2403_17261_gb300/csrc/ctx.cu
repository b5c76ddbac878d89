// ctx.cu -- the C ABI of libovl: context, scene upload, membership, and the
// timestep of Algorithm 1 as a sequence of kernels on one
// stream.  Counts that size the next buffers (contacts, graph edges,
// entries, pairs) are read back between phases; the load balance runs on the
// host between the graph and the membership phases.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <sstream>
#include <stdexcept>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "ctx.cuh"

using namespace ovl;

namespace ovl {

ovl_status check_device_status(ovl_ctx *c) {
    int s = read_i32(c, c->status.p);
    switch (s) {
        case DEV_OK: return OVL_OK;
        case DEV_ERR_CAPACITY:
            return fail(c, OVL_ERR_CAPACITY,
                        "a body touches more spheres of larger index than its neighbour capacity "
                        "(set from the radii: deep interpenetration)");
        case DEV_ERR_SLOTS: return fail(c, OVL_ERR_CAPACITY, "a worker holds 2^24 or more bodies");
        case DEV_ERR_NONFINITE: return fail(c, OVL_ERR_NONFINITE, "non-finite value in the blended state");
        case DEV_ERR_MEMBERSHIP:
            return fail(c, OVL_ERR_MEMBERSHIP, "dynamic body with no worker, or a worker index out of range");
        case DEV_ERR_COLOURS:
            return fail(c, OVL_ERR_CAPACITY, "a worker needs more than 128 colours (bodies in about 128 or more constraints)");
        case DEV_ERR_TIMEOUT:
            return fail(c, OVL_ERR_TIMEOUT, "a bounded device-side wait gave up (colouring rounds, or a tensor-core MMA)");
        default: return fail(c, OVL_ERR_CUDA, "unknown device status");
    }
}

}  // namespace ovl

namespace {

uint32_t next_pow2(uint64_t x) {
    uint32_t p = 1;
    while (p < x && p < (1u << 31)) p <<= 1;
    return p;
}

int bits_for(int n) {
    int b = 1;
    while ((1 << b) < n && b < 31) ++b;
    return b;
}

void mark(ovl_ctx *c, int i) {
    if (c->P.flags & OVL_FLAG_TIMING) CK(cudaEventRecord(c->ev[i], c->stream));
}

// ---- phases ----------------------------------------------------------------

// contact points and manifold indices (contexts with box bodies), else NULL
float4 *contact_points(ovl_ctx *c) { return c->has_boxes ? c->c_p.p : nullptr; }

void phase_contacts(ovl_ctx *c) {
    cudaStream_t s = c->stream;
    const int n = c->n;
    c->cell.ensure(n);
    c->bucket_count.ensure((size_t)c->tsize + 1);
    c->bucket_start.ensure((size_t)c->tsize + 1);
    c->cursor.ensure(c->tsize);
    c->items.ensure(n);
    c->nb_list.ensure((size_t)c->nb_total + 1);
    c->nb_count.ensure(n);
    c->ccount.ensure((size_t)n + 1);
    c->cstart.ensure((size_t)n + 1);
    CK(cudaMemsetAsync(c->bucket_count.p, 0, sizeof(int) * ((size_t)c->tsize + 1), s));
    CK(cudaMemsetAsync(c->cursor.p, 0, sizeof(int) * c->tsize, s));
    ContactArgs a{};
    a.st = c->st.p; a.im = c->im.p; a.n = n; a.sob = c->sob.p; a.scene_flags = c->scene_flags.p;
    a.inv_cs = 1.0f / c->cs; a.tmask = c->tsize - 1;
    a.cell = c->cell.p; a.bucket_count = c->bucket_count.p; a.bucket_start = c->bucket_start.p;
    a.cursor = c->cursor.p; a.items = c->items.p; a.planes = c->planes.p;
    a.plane_ptr = c->plane_ptr.p; a.plane_list = c->plane_list.p; a.margin = c->P.margin;
    a.nb_list = c->nb_list.p; a.nb_off = c->nb_off.p; a.nb_count = c->nb_count.p;
    a.contact_count = c->ccount.p;
    a.contact_start = c->cstart.p; a.status = c->status.p;
    a.half = c->has_boxes ? c->half.p : nullptr;
    launch_cells(a, s);
    scan_i32(c->bucket_count.p, c->bucket_start.p, (int)c->tsize, c->scan_tmp, s);
    launch_bucket_fill(a, s);
    launch_find_pairs(a, s);
    scan_i32(c->ccount.p, c->cstart.p, n, c->scan_tmp, s);
    c->nc = read_i32(c, c->cstart.p + n);
    c->c_ab.ensure(c->nc + 1);
    c->c_n.ensure(c->nc + 1);
    c->c_t1.ensure(c->nc + 1);
    if (c->has_boxes) c->c_p.ensure(c->nc + 1);
    a.c_ab = c->c_ab.p; a.c_n = c->c_n.p; a.c_t1 = c->c_t1.p;
    a.c_p = contact_points(c);
    launch_write_contacts(a, s);
}

void phase_graph(ovl_ctx *c) {
    cudaStream_t s = c->stream;
    const int n = c->n;
    c->deg.ensure((size_t)n + 1);
    c->tptr.ensure((size_t)n + 1);
    c->cursor2.ensure((size_t)n + 1);
    c->ucount.ensure((size_t)n + 1);
    c->row_ptr.ensure((size_t)n + 1);
    CK(cudaMemsetAsync(c->deg.p, 0, sizeof(int) * ((size_t)n + 1), s));
    CK(cudaMemsetAsync(c->cursor2.p, 0, sizeof(int) * ((size_t)n + 1), s));
    launch_edge_degree(c->c_ab.p, c->nc, c->jab.p, c->nj, c->im.p, n, c->deg.p, s);
    scan_i32(c->deg.p, c->tptr.p, n, c->scan_tmp, s);
    int e2 = read_i32(c, c->tptr.p + n);
    c->tcol.ensure((size_t)e2 + 1);
    launch_edge_fill(c->c_ab.p, c->nc, c->jab.p, c->nj, c->im.p, n, c->tptr.p, c->cursor2.p,
                     c->tcol.p, s);
    launch_adj_unique(c->tptr.p, n, c->tcol.p, c->ucount.p, s);
    scan_i32(c->ucount.p, c->row_ptr.p, n, c->scan_tmp, s);
    c->nadj = read_i32(c, c->row_ptr.p + n);
    c->col.ensure((size_t)c->nadj + 1);
    launch_adj_compact(c->tptr.p, c->tcol.p, n, c->row_ptr.p, c->col.p, s);
}

// Algorithm 6 on the host over the contacts between two dynamic bodies, in
// canonical order.  The GPU first compacts the contacts that can act: all
// dynamic pairs on removal steps, only worker-disjoint pairs otherwise.
void phase_load_balance(ovl_ctx *c, bool act, bool deact) {
    c->lb_candidates = 0;
    c->lb_host_ms = 0.0;
    if ((!act && !deact) || c->nc == 0) return;
    cudaStream_t s = c->stream;
    const int n = c->n;
    c->lb_flag.ensure(c->nc + 1);
    c->lb_pos.ensure(c->nc + 1);
    c->lb_pairs.ensure(c->nc + 1);
    const auto t0 = std::chrono::steady_clock::now();
    launch_lb_flags(c->c_ab.p, c->nc, c->im.p, n, c->mask.p, deact ? 0 : 1, c->lb_flag.p, contact_points(c), s);
    scan_i32(c->lb_flag.p, c->lb_pos.p, c->nc, c->scan_tmp, s);
    // the graph and the masks go to the host while the candidate count is read
    c->h_rp.ensure((size_t)n + 1);
    c->h_col.ensure((size_t)c->nadj + 1);
    c->h_mask.ensure(n);
    CK(cudaMemcpyAsync(c->h_rp.p, c->row_ptr.p, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->h_col.p, c->col.p, sizeof(int) * c->nadj, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->h_mask.p, c->mask.p, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, s));
    const int m = read_i32(c, c->lb_pos.p + c->nc);
    c->lb_candidates = m;
    if (m == 0) return;
    launch_lb_compact(c->c_ab.p, c->nc, c->lb_flag.p, c->lb_pos.p, c->lb_pairs.p, s);
    c->h_ab.ensure(m + 1);
    CK(cudaMemcpyAsync(c->h_ab.p, c->lb_pairs.p, sizeof(int2) * m, cudaMemcpyDeviceToHost, s));
    c->lb_loads.ensure((size_t)c->n_parts + 1);
    c->h_loads.ensure((size_t)c->n_parts + 1);
    const bool by_contacts = c->P.lb_load == OVL_LB_CONTACTS;
    if (by_contacts) {
        c->lb_deg.ensure((size_t)n + 1);
        c->h_deg.ensure((size_t)n + 1);
        launch_contact_degree(c->c_ab.p, c->nc, n, c->lb_deg.p, contact_points(c), s);
        CK(cudaMemcpyAsync(c->h_deg.p, c->lb_deg.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    }
    launch_worker_loads(c->mask.p, c->sob.p, c->part_base.p, by_contacts ? c->lb_deg.p : nullptr, n,
                        c->n_parts, c->lb_loads.p, s);
    CK(cudaMemcpyAsync(c->h_loads.p, c->lb_loads.p, sizeof(int) * c->n_parts, cudaMemcpyDeviceToHost, s));
    // the gamma-balls of the ends of the disjoint candidates, found on the
    // device (the pass activates those of its roots).  Not on removal steps:
    // there the activations come mostly from contacts that become disjoint
    // during the pass, and the host searches those (measured: no gain).
    const int *hb_start = nullptr, *hb_vtx = nullptr;
    if (act && !deact) {
        const int max_roots = (int)std::min<long long>(2LL * m, n);
        c->ball_root.ensure((size_t)n + 1);
        c->ball_size.ensure((size_t)n + 1);
        c->ball_start.ensure((size_t)n + 1);
        c->ball_list.ensure((size_t)max_roots + 1);
        CK(cudaMemsetAsync(c->ball_root.p, 0, sizeof(int) * ((size_t)n + 1), s));   // [n]: the root count
        CK(cudaMemsetAsync(c->ball_size.p, 0, sizeof(int) * n, s));
        int *const nroot = c->ball_root.p + n;
        launch_ball_roots(c->lb_pairs.p, m, c->mask.p, c->ball_root.p, c->ball_list.p, nroot, s);
        launch_balls(false, max_roots, c->ball_list.p, nroot, c->row_ptr.p, c->col.p, c->sob.p, c->scene_gamma.p,
                     c->ball_size.p, nullptr, nullptr, s);
        scan_i32(c->ball_size.p, c->ball_start.p, n, c->scan_tmp, s);
        const int total = read_i32(c, c->ball_start.p + n);
        c->ball_vtx.ensure((size_t)total + 1);
        launch_balls(true, max_roots, c->ball_list.p, nroot, c->row_ptr.p, c->col.p, c->sob.p, c->scene_gamma.p,
                     c->ball_size.p, c->ball_start.p, c->ball_vtx.p, s);
        c->h_ball_start.ensure((size_t)n + 1);
        c->h_ball_vtx.ensure((size_t)total + 1);
        CK(cudaMemcpyAsync(c->h_ball_start.p, c->ball_start.p, sizeof(int) * ((size_t)n + 1),
                           cudaMemcpyDeviceToHost, s));
        if (total) CK(cudaMemcpyAsync(c->h_ball_vtx.p, c->ball_vtx.p, sizeof(int) * (size_t)total,
                                      cudaMemcpyDeviceToHost, s));
        hb_start = c->h_ball_start.p;
        hb_vtx = c->h_ball_vtx.p;
    }
    CK(cudaStreamSynchronize(s));
    if ((int)c->lb_ws.size() != c->lb_threads) c->lb_ws.resize(c->lb_threads);
    host_load_balance(c->hs, c->h_mask.p, c->h_loads.p, by_contacts ? c->h_deg.p : nullptr, m, c->h_ab.p,
                      c->h_rp.p, c->h_col.p, act, deact, c->lb_ws, hb_start, hb_vtx);
    // no wait for the copy: the next kernels are ordered after it on s, and
    // the host touches h_mask again only after the next download into it
    CK(cudaMemcpyAsync(c->mask.p, c->h_mask.p, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
    c->lb_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

MemberArgs member_args(ovl_ctx *c) {
    MemberArgs a{};
    a.c_p = contact_points(c);
    a.n = c->n; a.nc = c->nc; a.nj = c->nj; a.n_parts = c->n_parts;
    a.im = c->im.p; a.sob = c->sob.p; a.n_sets = c->n_sets.p; a.part_base = c->part_base.p;
    a.joint_scene = c->joint_scene.p; a.mask = c->mask.p; a.c_ab = c->c_ab.p; a.jab = c->jab.p;
    a.entry_count = c->entry_count.p; a.entry_ptr = c->entry_ptr.p; a.entry_body = c->entry_body.p;
    a.entry_part = c->entry_part.p; a.entry_slot = c->entry_slot.p; a.part_list = c->part_list.p;
    a.part_bstart = c->part_bstart.p; a.cons_count = c->cons_count.p; a.cons_start = c->cons_start.p;
    a.pair_cons = c->pair_cons.p; a.pair_part = c->pair_part.p; a.ps_cons = c->ps_cons.p;
    a.ps_part = c->ps_part.p; a.part_pstart = c->part_pstart.p; a.p_key = c->p_key.p;
    a.p_slot = c->p_slot.p; a.p_lam0 = c->p_lam0.p; a.status = c->status.p;
    return a;
}

// stable grouping of items by a small key (< n_parts): out = item indices
void group_by(ovl_ctx *c, const int *key, int m, DBuf<int> &out) {
    cudaStream_t s = c->stream;
    c->sk.ensure(m + 1); c->sv.ensure(m + 1); c->sk2.ensure(m + 1); c->sv2.ensure(m + 1);
    out.ensure(m + 1);
    if (m == 0) return;
    CK(cudaMemcpyAsync(c->sk.p, key, sizeof(int) * m, cudaMemcpyDeviceToDevice, s));
    iota_u32(c->sv.p, m, s);
    bool alt = false;
    radix_sort_u32(c->sk.p, c->sv.p, c->sk2.p, c->sv2.p, m, bits_for(c->n_parts), c->sort_hist,
                   c->sort_tmp, s, &alt);
    CK(cudaMemcpyAsync(out.p, alt ? c->sv2.p : c->sv.p, sizeof(int) * m, cudaMemcpyDeviceToDevice, s));
}

void phase_membership(ovl_ctx *c, float dt_override) {
    (void)dt_override;
    cudaStream_t s = c->stream;
    const int n = c->n, P = c->n_parts;
    c->entry_count.ensure((size_t)n + 1);
    c->entry_ptr.ensure((size_t)n + 1);
    MemberArgs a = member_args(c);
    launch_entry_count(a, s);
    scan_i32(c->entry_count.p, c->entry_ptr.p, n, c->scan_tmp, s);
    c->ne = read_i32(c, c->entry_ptr.p + n);
    const int ne = c->ne;
    c->entry_body.ensure(ne + 1); c->entry_part.ensure(ne + 1); c->entry_slot.ensure(ne + 1);
    c->part_count.ensure((size_t)P + 1); c->part_bstart.ensure((size_t)P + 1);
    a = member_args(c);
    launch_entry_fill(a, s);
    group_by(c, c->entry_part.p, ne, c->part_list);
    CK(cudaMemsetAsync(c->part_count.p, 0, sizeof(int) * ((size_t)P + 1), s));
    histogram_i32(c->entry_part.p, ne, c->part_count.p, P, s);
    scan_i32(c->part_count.p, c->part_bstart.p, P, c->scan_tmp, s);
    a = member_args(c);
    launch_entry_slot(a, ne, s);
    // (worker, constraint) pairs
    const int K = c->nc + c->nj;
    c->cons_count.ensure((size_t)K + 1); c->cons_start.ensure((size_t)K + 1);
    a = member_args(c);
    launch_cons_count(a, s);
    scan_i32(c->cons_count.p, c->cons_start.p, K, c->scan_tmp, s);
    c->npairs = read_i32(c, c->cons_start.p + K);
    const int npr = c->npairs;
    c->pair_cons.ensure(npr + 1); c->pair_part.ensure(npr + 1); c->ps_cons.ensure(npr + 1);
    c->ps_part.ensure(npr + 1); c->part_pcount.ensure((size_t)P + 1); c->part_pstart.ensure((size_t)P + 1);
    c->p_key.ensure(npr + 1); c->p_slot.ensure(npr + 1); c->p_lam0.ensure(npr + 1);
    a = member_args(c);
    launch_pair_fill(a, s);
    DBuf<int> &order = c->pair_of_row;   // temporary use before colouring
    order.ensure(npr + 1);
    group_by(c, c->pair_part.p, npr, order);
    launch_pair_gather(a, reinterpret_cast<const uint32_t *>(order.p), npr, s);
    CK(cudaMemsetAsync(c->part_pcount.p, 0, sizeof(int) * ((size_t)P + 1), s));
    histogram_i32(c->pair_part.p, npr, c->part_pcount.p, P, s);
    scan_i32(c->part_pcount.p, c->part_pstart.p, P, c->scan_tmp, s);
    WarmArgs w{};
    w.ws_pstart = c->ws_pstart.p; w.ws_key = c->ws_key.p; w.ws_lam = c->ws_lam.p;
    w.factor = c->P.warmstart;
    launch_pair_setup(a, w, npr, s);
    // launch order of the per-worker kernels: most constraints first, so
    // the longest workers start in the first wave
    c->worker_order.ensure((size_t)P + 1);
    c->wk.ensure((size_t)P + 1); c->wk2.ensure((size_t)P + 1); c->wv2.ensure((size_t)P + 1);
    launch_worker_cost_keys(c->part_pstart.p, P, c->wk.p, c->worker_order.p, s);
    bool alt = false;
    radix_sort_u32(c->wk.p, c->worker_order.p, c->wk2.p, c->wv2.p, P, 24, c->sort_hist, c->sort_tmp, s, &alt);
    if (alt) std::swap(c->worker_order, c->wv2);
    // per-worker bodies and constraints on the host, for the launch plans
    c->h_pb.resize((size_t)P + 1);
    c->h_pp.resize((size_t)P + 1);
    download(c->h_pb.data(), c->part_bstart.p, (size_t)P + 1, s);
    download(c->h_pp.data(), c->part_pstart.p, (size_t)P + 1, s);
    CK(cudaStreamSynchronize(s));
    c->nb_max = 0;
    for (int p = 0; p < P; ++p) c->nb_max = std::max(c->nb_max, c->h_pb[p + 1] - c->h_pb[p]);
}

int colour_smem_capacity(ovl_ctx *c) {
    int avail = c->smem_optin - colour_static_smem() - 1024;
    int n = std::max(0, avail / 16);
    return c->P.smem_slot_limit > 0 ? std::min(n, c->P.smem_slot_limit) : n;
}

// CTAs per worker for the colouring: the smallest cluster whose share of the
// largest worker's slots fits one CTA's shared memory (16 B per slot)
void colour_config(ovl_ctx *c, int *cluster, int *slots) {
    const int cap = colour_smem_capacity(c);
    const int fixed = (c->P.pgs_cluster == 1 || c->P.pgs_cluster == 2 || c->P.pgs_cluster == 4 ||
                       c->P.pgs_cluster == 8) ? c->P.pgs_cluster : 0;
    for (int C = 1; C <= 8; C <<= 1) {
        if (fixed && C != fixed) continue;
        int per = std::max(1, (c->nb_max + C - 1) / C);
        if (per <= cap) { *cluster = C; *slots = per; return; }
    }
    *cluster = fixed ? fixed : 1;
    *slots = cap;
}

// Dynamic shared memory a solver CTA may use with 1 or 2 resident CTAs per SM
// (the solver's static shared memory -- row-bucket offsets, reductions -- is
// under 1 KB)
int solve_smem_budget(ovl_ctx *c, int ctas_per_sm) {
    return ctas_per_sm == 1 ? c->smem_optin - 2 * 1024 : (c->smem_per_sm / 2) - 3 * 1024;
}

// Shared-memory body slots per CTA (24 B each, the layout without masses: the
// CTA counts are planned with it, so adding the masses never adds CTAs), less
// the CTA's zero slot
int solve_slot_capacity(ovl_ctx *c, int ctas_per_sm) {
    int n = std::max(0, solve_smem_budget(c, ctas_per_sm) / solve_slot_bytes(false) - 1);
    return c->P.smem_slot_limit > 0 ? std::min(n, c->P.smem_slot_limit) : n;
}

// a launch keeps the masses in shared memory (32 B per slot) when its slots
// still fit that way
bool solve_masses_fit(ovl_ctx *c, int slots, int ctas_per_sm) {
    return c->P.smem_slot_limit <= 0 && solve_smem_bytes(slots, true) <= solve_smem_budget(c, ctas_per_sm);
}

// Per-worker CTA counts for the default launch: every worker starts at the
// fewest CTAs (1, 2, 3, 4, 6 or 8) whose shares of its bodies fit one CTA's
// shared memory; while all CTAs still fit the SMs, the worker with the most
// rows per CTA moves to the next count.  Workers with the same count form one launch, and
// the launches run side by side on the context's streams.  Every launch
// shape gives the same bits (no implicit FMA contraction in the solver),
// so the plan changes only the time.  Returns false when some worker does
// not fit even 8 CTAs (the uniform launch then takes it to global memory).
struct SolveClass { int C, first, count, slots; };

// the growth stops at this many CTAs per worker (more only where a
// worker's bodies need them), and leaves this many SMs unclaimed: clusters
// must fit inside one GPC, so a launch that claims every SM can leave a
// cluster waiting for a second wave
#ifndef OVL_SOLVE_MAX_GROW
#define OVL_SOLVE_MAX_GROW 4
#endif
#ifndef OVL_SOLVE_SM_SLACK
#define OVL_SOLVE_SM_SLACK 8
#endif

// CTA shapes of the per-class launches: threads, rows per thread, CTAs per SM
struct SolveShape { int threads, unroll, per_sm; };
constexpr SolveShape kSolveShapes[3] = {{512, 2, 1}, {512, 1, 2}, {256, 2, 2}};

// the shape without tuning: one CTA per SM while the workers do not
// outnumber the SMs, else two smaller CTAs per SM
// CTAs per worker the plans choose from (each a cluster size both the solver
// and the colouring are built for)
constexpr int kClusterSizes[] = {1, 2, 3, 4, 6, 8};

int default_solve_shape(const ovl_ctx *c) { return c->n_parts <= c->num_sms ? 0 : 2; }

// CTA count of every worker (shared by the colouring and the solve): the
// fewest of kClusterSizes whose shares of its bodies fit `cap` slots; then,
// while the total stays within `budget`, the worker with the most rows per
// CTA moves to the next size (at most OVL_SOLVE_MAX_GROW).  Empty if some
// worker needs more than 8.  (Sizes 5 and 7 were tried: the workers of the
// large pile need 1-4 CTAs each, so they changed no plan.)
std::vector<int> plan_worker_counts(ovl_ctx *c, int cap, long long budget) {
    const int P = c->n_parts;
    const std::vector<int> &pb = c->h_pb, &pp = c->h_pp;
    auto next = [](int k) { for (int x : kClusterSizes) if (x > k) return x; return 0; };
    std::vector<int> C(P);
    long long total = 0;
    for (int p = 0; p < P; ++p) {
        const int nb = pb[p + 1] - pb[p];
        int k = 1;
        while (k && (nb + k - 1) / k > cap) k = next(k);
        if (!k) return {};
        C[p] = k;
        total += k;
    }
    auto load = [&](int p) { return (double)(pp[p + 1] - pp[p]) / C[p]; };
    if (total <= budget) {
        std::vector<int> heap(P);
        std::iota(heap.begin(), heap.end(), 0);
        auto less = [&](int x, int y) { return load(x) < load(y) || (load(x) == load(y) && x > y); };
        std::make_heap(heap.begin(), heap.end(), less);
        while (!heap.empty()) {
            std::pop_heap(heap.begin(), heap.end(), less);
            const int p = heap.back();
            const int up = next(C[p]);
            if (!up || up > OVL_SOLVE_MAX_GROW || total + (up - C[p]) > budget) break;
            total += up - C[p];
            C[p] = up;
            std::push_heap(heap.begin(), heap.end(), less);
        }
    }
    return C;
}

// launch classes of a CTA-count plan: workers with equal counts, most CTAs
// first and longest first inside; the worker order goes to buf
void plan_classes_from(ovl_ctx *c, const std::vector<int> &C, std::vector<SolveClass> &classes,
                       DBuf<uint32_t> &buf) {
    const int P = c->n_parts;
    const std::vector<int> &pb = c->h_pb, &pp = c->h_pp;
    std::vector<int> order(P);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (C[x] != C[y]) return C[x] > C[y];
        return pp[x + 1] - pp[x] > pp[y + 1] - pp[y];
    });
    classes.clear();
    for (int i = 0; i < P; ++i) {
        const int p = order[i], nb = pb[p + 1] - pb[p];
        if (classes.empty() || classes.back().C != C[p]) classes.push_back({C[p], i, 0, 1});
        SolveClass &k = classes.back();
        k.count++;
        k.slots = std::max(k.slots, (nb + C[p] - 1) / C[p]);
    }
    std::vector<uint32_t> o(order.begin(), order.end());
    upload(buf, o.data(), o.size(), c->stream);
    c->h_class_C.assign(C.begin(), C.end());
}

bool plan_worker_classes(ovl_ctx *c, int cap, long long budget, std::vector<SolveClass> &classes,
                         DBuf<uint32_t> &buf) {
    const std::vector<int> C = plan_worker_counts(c, cap, budget);
    if (C.empty() && c->n_parts > 0) return false;
    plan_classes_from(c, C, classes, buf);
    return true;
}

// fewest CTAs of a plan before any growth (sum of the minimal counts)
long long fewest_ctas(ovl_ctx *c, int cap) {
    long long total = 0;
    for (int p = 0; p < c->n_parts; ++p) {
        const int nb = c->h_pb[p + 1] - c->h_pb[p];
        int k = 0;
        for (int x : kClusterSizes)
            if ((nb + x - 1) / x <= cap) { k = x; break; }
        if (!k) return -1;
        total += k;
    }
    return total;
}

// The per-worker plan keeps the masses in shared memory (32 B per body; two
// records per contact row, about 15 % less time per row) when the fewest CTAs
// that hold every worker that way fit the SMs at once, or when even 24 B per
// body (masses in the rows) needs several waves of CTAs (many small workers).
// Otherwise -- large workers that overflow one wave only slightly at 24 B per
// body -- it plans 24 B per body, and classes whose slots still fit take the
// masses.  (Measured on the large pile: planning 32 B per body past one wave
// made the solve up to 40 % slower than the 24 B plan.)
bool plan_solve_classes(ovl_ctx *c, const SolveShape &shape, std::vector<SolveClass> &classes) {
    const long long budget = (long long)shape.per_sm * c->num_sms - OVL_SOLVE_SM_SLACK;
    const long long slots = (long long)shape.per_sm * c->num_sms;
    const int cap_plain = solve_slot_capacity(c, shape.per_sm);
    int cap = cap_plain;
    if (c->P.smem_slot_limit <= 0) {
        const int cap_m = solve_smem_budget(c, shape.per_sm) / solve_slot_bytes(true) - 1;
        const long long with_m = fewest_ctas(c, cap_m), plain = fewest_ctas(c, cap_plain);
        if (with_m > 0 && (with_m <= slots || plain < 0 || plain > 2 * slots)) cap = cap_m;
    }
    const std::vector<int> C = plan_worker_counts(c, cap, budget);
    if (C.empty() && c->n_parts > 0) return false;
    plan_classes_from(c, C, classes, c->class_order);
    return true;
}

// The order in which a plan's classes are launched.  When all CTAs fit the
// SMs at once, classes of even cluster sizes go first, then odd ones, single
// CTAs last: clusters are placed in pairs of SMs more easily before odd
// clusters and single CTAs split the pairs (measured on the large pile: a
// plan of 32 three-CTA, 16 two-CTA and 16 one-CTA workers took 4.2 ms
// launched largest first and 2.5 ms this way).  A plan with more CTAs than
// SMs keeps the largest clusters first (the way measured faster there).
std::vector<size_t> class_launch_order(ovl_ctx *c, const std::vector<SolveClass> &classes) {
    std::vector<size_t> ord(classes.size());
    std::iota(ord.begin(), ord.end(), 0);
    long long ctas = 0;
    for (const SolveClass &k : classes) ctas += (long long)k.C * k.count;
    if (ctas > c->num_sms) return ord;
    auto key = [&](size_t k) { const int C = classes[k].C; return C == 1 ? 0 : (C % 2 == 0 ? 2 * 16 + C : 16 + C); };
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return key(x) > key(y); });
    return ord;
}

// launches class ord[j] (all classes when ord is empty) on side stream j
// (priorities falling with j), forked from and joined into the context's
// stream
template <class F>
void run_on_streams(ovl_ctx *c, size_t n, F &&launch, const std::vector<size_t> &ord = {}) {
    if (n > sizeof(c->aux) / sizeof(c->aux[0])) throw std::logic_error("more launch classes than side streams");
    if (n == 0) return;
    CK(cudaEventRecord(c->fork, c->stream));
    for (size_t j = 0; j < n; ++j) {
        const size_t k = ord.empty() ? j : ord[j];
        CK(cudaStreamWaitEvent(c->aux[j], c->fork, 0));
        launch(k, c->aux[j]);
    }
    for (size_t j = 0; j < n; ++j) {
        CK(cudaEventRecord(c->join[j], c->aux[j]));
        CK(cudaStreamWaitEvent(c->stream, c->join[j], 0));
    }
}

void launch_solve_classes(ovl_ctx *c, const SolveArgs &a, const SolveShape &shape,
                          const std::vector<SolveClass> &classes) {
    run_on_streams(c, classes.size(), [&](size_t k, cudaStream_t sk) {
        SolveArgs b = a;
        b.n_parts = classes[k].count;
        b.order = c->class_order.p + classes[k].first;
        b.smem_slots = classes[k].slots;
        launch_solve(b, shape.threads, classes[k].C, shape.unroll,
                     solve_masses_fit(c, classes[k].slots, shape.per_sm), sk);
    }, class_launch_order(c, classes));
}

void phase_colour(ovl_ctx *c) {
    const int P = c->n_parts, npr = c->npairs;
    c->p_colour.ensure(npr + 1);
    c->part_ncol.ensure((size_t)P + 1);
    c->part_rounds.ensure((size_t)P + 1);
    c->col_off.ensure((size_t)P * (2 * OVL_MAX_COLOURS + 1) + 1);
    c->pair_of_row.ensure(npr + 1);
    c->colour_scratch.ensure(3 * (size_t)c->ne + 1);
    c->worklist.ensure(npr + 1);
    c->worklist2.ensure(npr + 1);
    c->wprio.ensure(npr + 1);
    c->wprio2.ensure(npr + 1);
    ColourArgs a{};
    a.n_parts = P; a.part_bstart = c->part_bstart.p; a.part_pstart = c->part_pstart.p;
    a.order = c->worker_order.p;
    a.part_list = c->part_list.p; a.entry_body = c->entry_body.p;
    a.p_key = c->p_key.p; a.p_slot = c->p_slot.p; a.p_colour = c->p_colour.p;
    a.part_ncol = c->part_ncol.p; a.col_off = c->col_off.p; a.pair_of_row = c->pair_of_row.p;
    a.part_rounds = c->part_rounds.p;
    a.scratch = c->colour_scratch.p; a.hi_mask = c->colour_scratch.p + 2 * (size_t)c->ne;
    a.status = c->status.p;
    a.worklist = c->worklist.p; a.worklist2 = c->worklist2.p;
    a.wprio = c->wprio.p; a.wprio2 = c->wprio2.p;
    const bool fixed = c->P.pgs_cluster > 0 || c->P.smem_slot_limit > 0;
    std::vector<SolveClass> classes;
    if (!fixed && P > 0 &&
        plan_worker_classes(c, colour_smem_capacity(c), (long long)c->num_sms - OVL_SOLVE_SM_SLACK,
                            classes, c->colour_order)) {
        run_on_streams(c, classes.size(), [&](size_t k, cudaStream_t sk) {
            ColourArgs b = a;
            b.n_parts = classes[k].count;
            b.order = c->colour_order.p + classes[k].first;
            b.smem_slots = classes[k].slots;
            launch_colour(b, classes[k].C, sk);
        });
        return;
    }
    int cluster = 1, slots = 0;
    colour_config(c, &cluster, &slots);
    a.smem_slots = slots;
    launch_colour(a, cluster, c->stream);
}

void phase_rows(ovl_ctx *c, float dt_override) {
    const int npr = c->npairs;
    c->r0.ensure(npr + 1); c->r1.ensure(npr + 1); c->r2.ensure(npr + 1); c->r3.ensure(npr + 1);
    c->rpair.ensure(npr + 1); c->rlam.ensure(npr + 1);
    RowArgs a{};
    a.n = c->n; a.nc = c->nc; a.np = npr; a.pair_of_row = c->pair_of_row2.p; a.ps_cons = c->ps_cons.p;
    a.ps_part = c->ps_part.p; a.p_slot = c->p_slot.p; a.p_lam0 = c->p_lam0.p; a.c_ab = c->c_ab.p;
    a.c_n = c->c_n.p; a.c_t1 = c->c_t1.p; a.jab = c->jab.p; a.janc = c->janc.p;
    a.joint_scene = c->joint_scene.p; a.st = c->st.p; a.sob = c->sob.p; a.part_scene = c->part_scene.p;
    a.scene_dt = c->scene_dt.p; a.scene_mu = c->scene_mu.p; a.dt_override = dt_override;
    a.erp = c->P.erp; a.slop = c->P.slop;
    a.r0 = c->r0.p; a.r1 = c->r1.p; a.r2 = c->r2.p; a.r3 = c->r3.p; a.rlam = c->rlam.p;
    a.part_bstart = c->part_bstart.p; a.solve_C = c->solve_C.p; a.solve_M = c->solve_M.p;
    a.rpair = c->rpair.p; a.status = c->status.p;
    if (c->has_boxes) {
        c->row_full.ensure(npr + 1);
        c->rfull.ensure((size_t)FULL_ROW_WORDS * npr + 1);
        a.c_p = c->c_p.p; a.half = c->half.p; a.iib = c->iib.p;
        a.row_full = c->row_full.p; a.rfull = c->rfull.p;
    }
    launch_rows(a, c->stream);
}

// CTAs per worker (C) and shared-memory slots per CTA.  Preference: the
// smallest C for which every CTA of the launch is resident at once with two
// CTAs per SM (the largest worker's share fits half an SM's shared memory),
// then with one CTA per SM, so no worker waits for a second wave; otherwise
// the smallest C whose share fits one CTA.  A fixed pgs_cluster overrides C.
void solve_config(ovl_ctx *c, int *cluster, int *slots, int *unroll) {
    *unroll = 1;
    const int nbmax = c->nb_max;
    const int cap2 = solve_slot_capacity(c, 2), cap1 = solve_slot_capacity(c, 1);
    const int fixed = (c->P.pgs_cluster == 1 || c->P.pgs_cluster == 2 || c->P.pgs_cluster == 4 ||
                       c->P.pgs_cluster == 8) ? c->P.pgs_cluster : 0;
    // one resident CTA per SM with two rows per thread was the fastest shape
    // measured on the large pile; fall back to the others in order
    if (!fixed || fixed == 2) {
        const int per = (nbmax + 1) / 2;
        if (per <= cap1 && 2ll * c->n_parts <= c->num_sms) { *cluster = 2; *slots = std::max(per, 1); *unroll = 2; return; }
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int C = 1; C <= 8; C <<= 1) {
            if (fixed && C != fixed) continue;
            const int per = (nbmax + C - 1) / C;
            const long long ctas = (long long)c->n_parts * C;
            if (pass == 0 && per <= cap2 && ctas <= 2ll * c->num_sms) { *cluster = C; *slots = std::max(per, 1); return; }
            if (pass == 1 && per <= cap1 && ctas <= c->num_sms) { *cluster = C; *slots = std::max(per, 1); return; }
        }
    for (int C = 1; C <= 8; C <<= 1) {
        if (fixed && C != fixed) continue;
        const int per = (nbmax + C - 1) / C;
        if (per <= cap1) { *cluster = C; *slots = std::max(per, 1); return; }
    }
    // the largest workers go to the global-memory path
    *cluster = fixed ? fixed : 4;
    *slots = cap1;
}

int solve_threads(ovl_ctx *c) {
    int t = c->P.pgs_threads;
    if (t <= 0) t = 512;
    t = std::max(32, std::min(1024, (t + 31) / 32 * 32));
    return t;
}

SolveArgs solve_args(ovl_ctx *c, float dt_override, int iters) {
    SolveArgs a{};
    a.n_parts = c->n_parts; a.part_bstart = c->part_bstart.p; a.part_list = c->part_list.p;
    a.order = c->worker_order.p;
    a.entry_body = c->entry_body.p; a.part_ncol = c->part_ncol.p; a.col_off = c->col_off2.p;
    a.part_scene = c->part_scene.p; a.scene_dt = c->scene_dt.p; a.dt_override = dt_override;
    a.gravity = make_float3(c->P.gravity[0], c->P.gravity[1], c->P.gravity[2]);
    a.st = c->st.p; a.r0 = c->r0.p; a.r1 = c->r1.p; a.r2 = c->r2.p; a.r3 = c->r3.p;
    a.rlam = c->rlam.p;
    a.rpair = c->rpair.p; a.scene_mu = c->scene_mu.p; a.n_entries = c->ne;
    a.lam_out = c->lam_out.p; a.copies = c->copies.p; a.scratch = c->solve_scratch.p;
    a.iters = iters; a.flags = c->P.flags;
    a.res_tol = c->P.res_tol; a.res_check_every = c->P.res_check_every;
    a.part_iters = c->part_iters.p; a.part_res_sq = c->part_res_sq.p; a.status = c->status.p;
    if (c->has_boxes) { a.row_full = c->row_full.p; a.rfull = c->rfull.p; }
    return a;
}

// problem-size bucket of the autotuner: the number of workers and the largest
// worker's body count rounded up to a power of four
std::string tune_key(ovl_ctx *c) {
    int b = 1;
    while (b < c->nb_max) b <<= 2;
    std::ostringstream k;
    k << "P" << c->n_parts << "_nb" << b;
    return k.str();
}

// shared-memory slots for a cluster size (the largest worker's share), or 0
// if that share does not fit one CTA
int solve_slots_for(ovl_ctx *c, int cluster) {
    int per = std::max(1, (c->nb_max + cluster - 1) / cluster);
    return per <= solve_slot_capacity(c, 1) ? per : 0;
}

// K13: time every feasible uniform launch (CTAs per worker, threads per CTA,
// rows per thread and colour step) and every per-worker plan shape on this
// step's rows and keep the fastest for the bucket.
// Rows of one colour are independent, so every candidate computes the same
// bits; re-running the row build restores the warm-start impulses.
// How this step's solve is launched: per-worker classes (shape >= 0) or one
// uniform launch.
struct SolvePlan {
    int shape = -1;
    std::vector<SolveClass> classes;
    int cluster = 1, threads = 512, unroll = 1, slots = 0;
};

// Every worker's CTA count goes to the device and the rows of every colour
// are regrouped by the CTA that owns them (it holds the row's first dynamic
// body); the row build then follows that order.
void apply_solve_order(ovl_ctx *c, const SolvePlan &pl) {
    const int P = c->n_parts;
    std::vector<int> C(P, pl.cluster);
    if (pl.shape >= 0) C = c->h_class_C;
    upload(c->solve_C, C.data(), (size_t)P, c->stream);
    // which workers' launches keep the masses in shared memory (their rows
    // take the packed form); the classes of a per-worker plan differ in C
    std::vector<int> M(P, 0);
    if (pl.shape >= 0) {
        const int per_sm = kSolveShapes[pl.shape].per_sm;
        for (int p = 0; p < P; ++p)
            for (const SolveClass &k : pl.classes)
                if (k.C == C[p]) M[p] = solve_masses_fit(c, k.slots, per_sm) ? 1 : 0;
    } else {
        std::fill(M.begin(), M.end(), solve_masses_fit(c, pl.slots, solve_ctas_per_sm(pl.unroll)) ? 1 : 0);
    }
    upload(c->solve_M, M.data(), (size_t)P, c->stream);
    c->col_off2.ensure((size_t)P * OWNER_NB + 1);
    c->pair_of_row2.ensure((size_t)c->npairs + 1);
    c->row_owner.ensure((size_t)c->npairs + 1);
    launch_row_owner(P, c->part_bstart.p, c->part_ncol.p, c->solve_C.p, c->col_off.p, c->pair_of_row.p,
                     c->p_slot.p, c->row_owner.p, c->pair_of_row2.p, c->col_off2.p, c->stream);
}

void launch_solve_plan(ovl_ctx *c, const SolvePlan &pl, float dt_override, int iters) {
    const int P = c->n_parts, npr = c->npairs;
    c->lam_out.ensure(npr + 1);
    c->copies.ensure(4 * (size_t)c->ne + 1);
    c->solve_scratch.ensure(2 * (size_t)c->ne + 1);
    c->part_iters.ensure((size_t)P + 1);
    c->part_res_sq.ensure((size_t)P + 1);
    CK(cudaMemsetAsync(c->part_res_sq.p, 0, sizeof(double) * ((size_t)P + 1), c->stream));
    SolveArgs a = solve_args(c, dt_override, iters);
    c->last_ctas = c->last_ctas_masses = 0;
    if (pl.shape >= 0) {
        launch_solve_classes(c, a, kSolveShapes[pl.shape], pl.classes);
        for (const SolveClass &k : pl.classes) {
            c->last_ctas += (long long)k.C * k.count;
            if (solve_masses_fit(c, k.slots, kSolveShapes[pl.shape].per_sm)) c->last_ctas_masses += (long long)k.C * k.count;
        }
        c->last_cluster = pl.classes.front().C;
        c->last_plan_per_worker = true;
        c->last_threads = kSolveShapes[pl.shape].threads;
        c->last_unroll = kSolveShapes[pl.shape].unroll;
        return;
    }
    a.smem_slots = pl.slots;
    const bool masses = solve_masses_fit(c, pl.slots, solve_ctas_per_sm(pl.unroll));
    launch_solve(a, pl.threads, pl.cluster, pl.unroll, masses, c->stream);
    c->last_ctas = (long long)pl.cluster * P;
    c->last_ctas_masses = masses ? c->last_ctas : 0;
    c->last_cluster = pl.cluster;
    c->last_plan_per_worker = false;
    c->last_threads = pl.threads;
    c->last_unroll = pl.unroll;
}

// K13: time every feasible uniform launch (CTAs per worker, threads per CTA,
// rows per thread and colour step) and every per-worker plan shape on this
// step's rows and keep the fastest for the bucket.  Rows of one colour are
// independent, so every candidate computes the same bits; rebuilding the
// rows restores the warm-start impulses.
void autotune(ovl_ctx *c, float dt_override, int iters, const std::string &key) {
    cudaStream_t s = c->stream;
    ovl_ctx::TuneCfg best{0, 0, 0, 1e30f, 0};
    cudaEvent_t e0 = c->ev[10], e1 = c->ev[11];
    auto time_plan = [&](const SolvePlan &pl) {
        apply_solve_order(c, pl);
        phase_rows(c, dt_override);
        CK(cudaEventRecord(e0, s));
        launch_solve_plan(c, pl, dt_override, iters);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
    };
    for (int cl : {1, 2, 4, 8})
        for (int th : {256, 512})
            for (int un : {1, 2}) {
                SolvePlan pl;
                pl.cluster = cl; pl.threads = th; pl.unroll = un;
                pl.slots = solve_slots_for(c, cl);
                if (!pl.slots) continue;
                const float ms = time_plan(pl);
                if (ms < best.ms) best = {cl, th, un, ms, 0};
            }
    for (int sh = 0; sh < 3; ++sh) {
        SolvePlan pl;
        if (!plan_solve_classes(c, kSolveShapes[sh], pl.classes)) continue;
        pl.shape = sh;
        const float ms = time_plan(pl);
        if (ms < best.ms) best = {0, kSolveShapes[sh].threads, kSolveShapes[sh].unroll, ms, sh + 1};
    }
    if (best.cluster || best.shape) c->tuned[key] = best;
}

// The launch of this step's solve: the autotuner's choice for the bucket
// (OVL_FLAG_AUTOTUNE), else the per-worker plan with the default shape, else
// (fixed shapes, or workers too large for 8 CTAs) one uniform launch.
SolvePlan plan_solve(ovl_ctx *c, float dt_override, int iters) {
    const int P = c->n_parts;
    SolvePlan pl;
    pl.threads = solve_threads(c);
    const bool fixed = c->P.pgs_cluster > 0 || c->P.pgs_threads > 0 || c->P.smem_slot_limit > 0;
    int shape = fixed ? -1 : default_solve_shape(c);
    bool tuned_uniform = false;
    if (!fixed && (c->P.flags & OVL_FLAG_AUTOTUNE) && P > 0) {
        std::string key = tune_key(c);
        auto it = c->tuned.find(key);
        if (it == c->tuned.end()) {
            autotune(c, dt_override, iters, key);
            it = c->tuned.find(key);
        }
        if (it != c->tuned.end()) {
            if (it->second.shape > 0) {
                shape = it->second.shape - 1;
            } else if (int sl = solve_slots_for(c, it->second.cluster)) {
                shape = -1;
                pl.cluster = it->second.cluster;
                pl.threads = it->second.threads;
                pl.unroll = it->second.unroll;
                pl.slots = sl;
                tuned_uniform = true;
            }
        }
    }
    if (shape >= 0 && P > 0 && plan_solve_classes(c, kSolveShapes[shape], pl.classes)) {
        pl.shape = shape;
        return pl;
    }
    if (!tuned_uniform) solve_config(c, &pl.cluster, &pl.slots, &pl.unroll);
    return pl;
}

// The geodesic phase is 2 beta + 4 small launches whose arguments change only
// when a buffer is reallocated or the entry count changes, so it is captured
// once as a CUDA graph and replayed while they stay the same.
void enqueue_geodesics(ovl_ctx *c, cudaStream_t s) {
    CK(cudaMemsetAsync(c->visited.p, 0, sizeof(uint32_t) * ((size_t)((c->vb_bits + 31) / 32) + 1), s));
    CK(cudaMemsetAsync(c->qctl.p, 0, sizeof(int) * ((size_t)c->beta_max + 4), s));
    fill_u8(c->D.p, 255, c->D.cap, s);   // the whole buffer: the graph then outlives entry counts
    GeoArgs a{};
    a.n = c->n; a.mask = c->mask.p; a.sob = c->sob.p; a.scene_beta = c->scene_beta.p;
    a.body_base = c->body_base.p; a.vb_base = c->vb_base.p; a.row_ptr = c->row_ptr.p; a.col = c->col.p;
    a.entry_ptr = c->entry_ptr.p; a.visited = c->visited.p; a.queue = c->queue.p; a.qctl = c->qctl.p;
    a.D = c->D.p;
    launch_geo_sources(a, s);
    for (int L = 1; L <= c->beta_max; ++L) launch_geo_level(a, L, s);
}

// s: the stream the weights are computed on
void phase_geodesics(ovl_ctx *c, cudaStream_t s) {
    c->D.ensure(c->ne + 1);
    c->visited.ensure((size_t)((c->vb_bits + 31) / 32) + 1);
    c->queue.ensure((size_t)c->vb_bits + 1);
    c->qctl.ensure((size_t)c->beta_max + 4);
    const std::vector<const void *> key = {
        c->D.p, c->visited.p, c->queue.p, c->qctl.p, c->mask.p, c->row_ptr.p, c->col.p,
        c->entry_ptr.p, c->sob.p, c->scene_beta.p, c->body_base.p, c->vb_base.p,
        (const void *)(intptr_t)c->D.cap, (const void *)(intptr_t)c->n, (const void *)(intptr_t)c->beta_max,
        (const void *)(intptr_t)c->vb_bits};
    if (!c->geo_exec || key != c->geo_key) {
        if (c->geo_exec) { cudaGraphExecDestroy(c->geo_exec); c->geo_exec = nullptr; }
        const long long l0 = launch_count();
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_geodesics(c, s);
        } catch (...) {
            cudaGraph_t partial = nullptr;
            cudaStreamEndCapture(s, &partial);   // leave the stream usable
            if (partial) cudaGraphDestroy(partial);
            throw;
        }
        CK(cudaStreamEndCapture(s, &g));
        cudaError_t e = cudaGraphInstantiate(&c->geo_exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        c->geo_key = key;
        c->geo_kernels = launch_count() - l0;
        note_launches(-c->geo_kernels);   // counted when replayed below
    }
    CK(cudaGraphLaunch(c->geo_exec, s));
    note_launches(c->geo_kernels);
}

void phase_blend(ovl_ctx *c, float dt_override) {
    c->weight.ensure(c->ne + 1);
    c->st_alt.ensure(4 * (size_t)c->n);
    BlendArgs a{};
    a.n = c->n; a.entry_ptr = c->entry_ptr.p; a.D = c->D.p; a.copies = c->copies.p; a.st_in = c->st.p;
    a.st_out = c->st_alt.p; a.weight = c->weight.p; a.status = c->status.p;
    a.sob = c->sob.p; a.scene_dt = c->scene_dt.p; a.dt_override = dt_override;
    a.uniform = c->P.weights == OVL_WEIGHTS_UNIFORM;
    launch_blend(a, c->stream);
    std::swap(c->st, c->st_alt);
    // the impulses of this step become the next step's warm-start cache
    std::swap(c->ws_key, c->p_key);
    std::swap(c->ws_lam, c->lam_out);
    std::swap(c->ws_pstart, c->part_pstart);
    c->ws_n = c->npairs;
}

ovl_status run_step(ovl_ctx *c, float dt, int iters) {
    if (!c->has_scene) return fail(c, OVL_ERR_ARG, "no scene uploaded");
    if (iters < 0) return fail(c, OVL_ERR_ARG, "iters must be >= 0");
    cudaStream_t s = c->stream;
    const long long launches0 = launch_count();
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(int), s));
    bool deact = c->P.lb_deact_every > 0 && (c->step_index % c->P.lb_deact_every) == 0;
    mark(c, 0);
    phase_contacts(c);
    mark(c, 1);
    phase_graph(c);
    mark(c, 2);
    phase_load_balance(c, c->P.lb_activate != 0, deact);
    mark(c, 3);
    phase_membership(c, dt);
    phase_warmstart(c, dt);
    // The geodesic weights need only the membership and the graph.  When the
    // workers do not outnumber the SMs (the solve is one wave), they run on
    // their own stream while the colouring and the solve proceed, and the
    // blend waits for them; with more workers the solve's waves would lose
    // SMs to them, so they run after the solve.
    const bool geo_beside = c->n_parts <= c->num_sms;
    cudaStream_t gs = geo_beside ? c->geo_stream : s;
    auto geodesics = [&]() {
        if (geo_beside) {
            CK(cudaEventRecord(c->geo_fork, s));
            CK(cudaStreamWaitEvent(c->geo_stream, c->geo_fork, 0));
        }
        if (c->P.flags & OVL_FLAG_TIMING) CK(cudaEventRecord(c->ev[14], gs));
        phase_geodesics(c, gs);
        if (c->P.flags & OVL_FLAG_TIMING) CK(cudaEventRecord(c->ev[15], gs));
        if (geo_beside) CK(cudaEventRecord(c->geo_join, c->geo_stream));
    };
    if (geo_beside) geodesics();
    mark(c, 4);
    phase_colour(c);
    mark(c, 5);
    const SolvePlan plan = plan_solve(c, dt, iters);
    apply_solve_order(c, plan);
    phase_rows(c, dt);
    mark(c, 6);
    launch_solve_plan(c, plan, dt, iters);
    phase_log(c);
    mark(c, 7);
    if (geo_beside) CK(cudaStreamWaitEvent(s, c->geo_join, 0));
    else geodesics();
    mark(c, 8);
    phase_blend(c, dt);
    mark(c, 9);
    ovl_status st = check_device_status(c);
    c->last_launches = launch_count() - launches0;
    c->have_step = true;
    if (c->P.flags & OVL_FLAG_TIMING) {
        CK(cudaEventSynchronize(c->ev[9]));
        for (int i = 0; i < 9; ++i) CK(cudaEventElapsedTime(&c->phase_ms[i], c->ev[i], c->ev[i + 1]));
        // geodesics: their own stream's time (they overlap colouring and solve)
        CK(cudaEventElapsedTime(&c->phase_ms[7], c->ev[14], c->ev[15]));
        CK(cudaEventElapsedTime(&c->phase_ms[9], c->ev[0], c->ev[9]));
        c->phase_ms[10] = 0.f;
        if (c->feat_valid) CK(cudaEventElapsedTime(&c->phase_ms[10], c->ev[12], c->ev[13]));
    }
    if (st != OVL_OK) return st;
    c->step_index++;
    return OVL_OK;
}

void validate_masks(const ovl_ctx *c, const uint64_t *m) {
    for (int b = 0; b < c->n; ++b) {
        int ns = c->hs.n_sets[c->hs.sob[b]];
        uint64_t allowed = ns >= 64 ? ~0ull : ((1ull << ns) - 1ull);
        bool dyn = c->h_im[b] > 0.f;
        if ((dyn && m[b] == 0) || (!dyn && m[b] != 0) || (m[b] & ~allowed))
            throw std::invalid_argument("membership: body " + std::to_string(b) +
                                        " has an empty or out-of-range worker mask");
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

ovl_status ovl_default_params(ovl_params *p) {
    if (!p) return OVL_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->gravity[0] = 0.f; p->gravity[1] = 0.f; p->gravity[2] = -9.81f;
    p->margin = 0.05f; p->erp = 0.2f; p->slop = 0.001f; p->warmstart = 1.0f;
    p->lb_activate = 1; p->lb_deact_every = 1;
    p->res_tol = 0.f; p->res_check_every = 0; p->pgs_threads = 0; p->flags = 0;
    return OVL_OK;
}

ovl_status ovl_create(ovl_ctx **out, const ovl_params *p, void *cuda_stream) {
    if (!out) return OVL_ERR_ARG;
    *out = nullptr;
    ovl_ctx *c = new (std::nothrow) ovl_ctx();
    if (!c) return OVL_ERR_ARG;
    if (p) c->P = *p; else ovl_default_params(&c->P);
    if ((c->P.lb_load != OVL_LB_BODIES && c->P.lb_load != OVL_LB_CONTACTS) ||
        (c->P.weights != OVL_WEIGHTS_GEODESIC && c->P.weights != OVL_WEIGHTS_UNIFORM)) {
        delete c;
        return OVL_ERR_ARG;
    }
    // The per-class launches use up to seven streams.  With CUDA's default
    // of 8 hardware work queues per device, streams created elsewhere in the
    // process make some of them share a queue, and launches on a shared queue
    // run one after another (measured: the 512-scene batch's solve 4.4 ms
    // instead of 3.4 ms).  The setting is read when the process's CUDA
    // context is created, so it only helps if that has not happened yet.
    setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0);
    ovl_status st = guarded(c, [&]() -> ovl_status {
        CK(cudaGetDevice(&c->device));
        CK(cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
        CK(cudaDeviceGetAttribute(&c->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
        mlp_kernels_setup(c->device);
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        for (auto &e : c->ev) CK(cudaEventCreate(&e));
        // the class launched first gets the highest priority, so that when a
        // plan has more CTAs than SMs its CTAs are placed before the later
        // classes' (numerically lower is higher)
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int j = 0; j < (int)(sizeof(c->aux) / sizeof(c->aux[0])); ++j)
            CK(cudaStreamCreateWithPriority(&c->aux[j], cudaStreamNonBlocking, std::min(least, greatest + j)));
        CK(cudaStreamCreateWithFlags(&c->geo_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->geo_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->geo_join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
        for (auto &e : c->join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->lb_threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        c->status.ensure(4);
        CK(cudaMemsetAsync(c->status.p, 0, 4 * sizeof(int), c->stream));
        return OVL_OK;
    });
    if (st != OVL_OK) {
        delete c;
        return st;
    }
    *out = c;
    return OVL_OK;
}

const char *ovl_last_error(const ovl_ctx *c) { return c ? c->err.c_str() : "null context"; }

const char *ovl_phase_name(int32_t phase) {
    static const char *names[] = {"contacts", "graph",     "load_balance", "membership",
                                  "colouring", "rows",     "solve",        "geodesics",
                                  "blend",     "total",    "warmstart"};
    return (phase >= 0 && phase < 11) ? names[phase] : "";
}

}  // extern "C"

namespace {

void release_all(ovl_ctx *c) {
    c->st.release(); c->st_alt.release(); c->radius.release(); c->im.release();
    c->scene_mu.release(); c->scene_dt.release(); c->sob.release(); c->scene_flags.release();
    c->n_sets.release(); c->part_base.release(); c->body_base.release(); c->scene_beta.release(); c->scene_gamma.release();
    c->joint_scene.release(); c->part_scene.release(); c->planes.release(); c->plane_ptr.release();
    c->plane_list.release(); c->jab.release(); c->janc.release(); c->vb_base.release();
    c->mask.release(); c->cell.release(); c->bucket_count.release(); c->bucket_start.release();
    c->cursor.release(); c->items.release(); c->nb_list.release(); c->nb_count.release(); c->nb_off.release();
    c->ccount.release(); c->cstart.release(); c->c_ab.release(); c->c_n.release(); c->c_t1.release();
    c->deg.release(); c->tptr.release(); c->cursor2.release(); c->tcol.release(); c->ucount.release();
    c->row_ptr.release(); c->col.release(); c->entry_count.release(); c->entry_ptr.release();
    c->entry_body.release(); c->entry_part.release(); c->entry_slot.release(); c->part_list.release();
    c->part_count.release(); c->part_bstart.release(); c->sk.release(); c->sv.release();
    c->sk2.release(); c->sv2.release(); c->cons_count.release(); c->cons_start.release();
    c->pair_cons.release(); c->pair_part.release(); c->ps_cons.release(); c->ps_part.release();
    c->part_pcount.release(); c->part_pstart.release(); c->p_colour.release(); c->part_ncol.release(); c->part_rounds.release();
    c->col_off.release(); c->pair_of_row.release(); c->p_key.release(); c->p_slot.release();
    c->p_lam0.release(); c->colour_scratch.release(); c->worklist.release(); c->worklist2.release(); c->wprio.release(); c->wprio2.release(); c->r0.release(); c->r1.release();
    c->r2.release(); c->rlam.release(); c->lam_out.release(); c->r3.release(); c->rpair.release(); c->ws_pstart.release();
    c->ws_key.release(); c->ws_lam.release(); c->copies.release(); c->solve_scratch.release();
    c->part_iters.release(); c->part_res_sq.release(); c->visited.release(); c->queue.release();
    c->qctl.release(); c->D.release(); c->weight.release(); c->stage13.release(); c->scan_tmp.release();
    c->sort_hist.release(); c->sort_tmp.release();
    c->lb_flag.release(); c->lb_pos.release(); c->lb_pairs.release();
    c->ball_root.release(); c->ball_size.release(); c->ball_start.release(); c->ball_vtx.release();
    c->ball_list.release();
    c->worker_order.release(); c->wk.release(); c->wk2.release(); c->wv2.release();
    c->class_order.release(); c->colour_order.release(); c->solve_C.release(); c->solve_M.release(); c->col_off2.release();
    c->row_owner.release();
    c->pair_of_row2.release(); c->lb_loads.release();
    c->half.release(); c->iib.release(); c->c_p.release(); c->row_full.release(); c->rfull.release();
}


void reset_warmstart(ovl_ctx *c) {
    c->ws_pstart.ensure((size_t)c->n_parts + 1);
    CK(cudaMemsetAsync(c->ws_pstart.p, 0, sizeof(int) * ((size_t)c->n_parts + 1), c->stream));
    c->ws_key.ensure(1);
    c->ws_lam.ensure(1);
    c->ws_n = 0;
}

void upload_masks(ovl_ctx *c, const std::vector<uint64_t> &m) {
    upload(c->mask, m.data(), m.size(), c->stream);
    CK(cudaStreamSynchronize(c->stream));
}

std::vector<uint64_t> download_masks(ovl_ctx *c) {
    std::vector<uint64_t> m(c->n);
    if (c->n) CK(cudaMemcpyAsync(m.data(), c->mask.p, sizeof(uint64_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return m;
}


}  // namespace

extern "C" {

ovl_status ovl_destroy(ovl_ctx *c) {
    if (!c) return OVL_ERR_ARG;
    if (c->stream) cudaStreamSynchronize(c->stream);
    release_all(c);
    release_mlp(c);
    c->h_loads.release();
    c->h_ball_start.release(); c->h_ball_vtx.release();
    c->h_i32.release(); c->h_ab.release(); c->h_rp.release(); c->h_col.release(); c->h_mask.release();
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &x : c->aux)
        if (x) { cudaStreamSynchronize(x); cudaStreamDestroy(x); }
    if (c->geo_stream) { cudaStreamSynchronize(c->geo_stream); cudaStreamDestroy(c->geo_stream); }
    if (c->geo_fork) cudaEventDestroy(c->geo_fork);
    if (c->geo_join) cudaEventDestroy(c->geo_join);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->geo_exec) cudaGraphExecDestroy(c->geo_exec);
    for (auto &e : c->join)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return OVL_OK;
}

ovl_status ovl_scene_upload(ovl_ctx *c, const ovl_scene_desc *d) {
    return guarded(c, [&]() -> ovl_status {
        if (!d || d->n_bodies <= 0 || !d->state || !d->radius || !d->inv_mass)
            return fail(c, OVL_ERR_ARG, "scene: bodies, state, radius and inv_mass are required");
        const int n = d->n_bodies, ns = d->n_scenes > 0 ? d->n_scenes : 1;
        if (n >= (1 << 26)) return fail(c, OVL_ERR_ARG, "scene: at most 2^26 - 1 bodies");
        if (d->n_planes < 0 || d->n_joints < 0) return fail(c, OVL_ERR_ARG, "scene: negative counts");
        if (d->n_planes > 0 && !d->planes) return fail(c, OVL_ERR_ARG, "scene: planes missing");
        if (d->n_joints > 0 && (!d->joint_bodies || !d->joint_anchors))
            return fail(c, OVL_ERR_ARG, "scene: joints missing");
        if (!d->scene_mu || !d->scene_dt || !d->scene_flags || !d->scene_gamma || !d->scene_beta || !d->n_sets)
            return fail(c, OVL_ERR_ARG, "scene: per-scene arrays are required");
        // boxes: extents finite and >= 0; a box's radius bounds it (the broad
        // phase tests bounding spheres)
        bool boxes = false;
        if (d->half_extents)
            for (int b = 0; b < n; ++b) {
                const float *h = d->half_extents + 3 * (size_t)b;
                for (int k = 0; k < 3; ++k)
                    if (!(h[k] >= 0.f) || !std::isfinite(h[k]))
                        return fail(c, OVL_ERR_ARG, "scene: half extents must be finite and >= 0");
                if (h[0] > 0.f || h[1] > 0.f || h[2] > 0.f) {
                    boxes = true;
                    const double hh = std::sqrt((double)h[0] * h[0] + (double)h[1] * h[1] + (double)h[2] * h[2]);
                    if ((double)d->radius[b] < hh * (1.0 - 1e-6))
                        return fail(c, OVL_ERR_ARG, "scene: a box's radius must bound it (>= |half extents|)");
                }
            }
        std::vector<int> sob(n, 0);
        if (d->scene_of_body) std::copy(d->scene_of_body, d->scene_of_body + n, sob.begin());
        for (int b = 0; b < n; ++b) {
            if (sob[b] < 0 || sob[b] >= ns || (b > 0 && sob[b] < sob[b - 1]))
                return fail(c, OVL_ERR_ARG, "scene: scene_of_body must be non-decreasing and < n_scenes");
            if (!(d->radius[b] > 0.f) || !(d->inv_mass[b] >= 0.f))
                return fail(c, OVL_ERR_ARG, "scene: radius must be > 0 and inv_mass >= 0");
        }
        for (int s = 0; s < ns; ++s) {
            if (d->n_sets[s] < 1 || d->n_sets[s] > 64) return fail(c, OVL_ERR_ARG, "scene: n_sets must be 1..64");
            if (d->scene_beta[s] < 0 || d->scene_beta[s] > 254 || d->scene_gamma[s] < 0)
                return fail(c, OVL_ERR_ARG, "scene: beta must be 0..254 and gamma >= 0");
            if (!(d->scene_dt[s] > 0.f)) return fail(c, OVL_ERR_ARG, "scene: dt must be > 0");
        }
        cudaStream_t s = c->stream;
        CK(cudaStreamSynchronize(s));
        release_all(c);
        c->status.ensure(4);
        c->n = n; c->ns = ns; c->np = d->n_planes; c->nj = d->n_joints;
        c->h_radius.assign(d->radius, d->radius + n);
        c->h_im.assign(d->inv_mass, d->inv_mass + n);
        // scene ranges and worker numbering
        c->h_body_base.assign(ns + 1, 0);
        for (int b = 0; b < n; ++b) c->h_body_base[sob[b] + 1]++;
        for (int i = 0; i < ns; ++i) c->h_body_base[i + 1] += c->h_body_base[i];
        std::vector<int> part_base(ns + 1, 0);
        for (int i = 0; i < ns; ++i) part_base[i + 1] = part_base[i] + d->n_sets[i];
        c->n_parts = part_base[ns];
        c->h_part_scene.assign(c->n_parts, 0);
        for (int i = 0; i < ns; ++i)
            for (int w = 0; w < d->n_sets[i]; ++w) c->h_part_scene[part_base[i] + w] = i;
        std::vector<long long> vb(ns + 1, 0);
        for (int i = 0; i < ns; ++i)
            vb[i + 1] = vb[i] + (long long)d->n_sets[i] * (c->h_body_base[i + 1] - c->h_body_base[i]);
        c->vb_bits = vb[ns];
        c->beta_max = 0;
        for (int i = 0; i < ns; ++i) c->beta_max = std::max(c->beta_max, d->scene_beta[i]);
        // planes grouped by scene
        std::vector<int> pscene(c->np, 0);
        if (d->plane_scene) std::copy(d->plane_scene, d->plane_scene + c->np, pscene.begin());
        c->h_plane_ptr.assign(ns + 1, 0);
        for (int p = 0; p < c->np; ++p) {
            if (pscene[p] < 0 || pscene[p] >= ns) return fail(c, OVL_ERR_ARG, "scene: bad plane_scene");
            c->h_plane_ptr[pscene[p] + 1]++;
        }
        for (int i = 0; i < ns; ++i) c->h_plane_ptr[i + 1] += c->h_plane_ptr[i];
        std::vector<int> plist(c->np), pfill(c->h_plane_ptr.begin(), c->h_plane_ptr.end() - 1);
        for (int p = 0; p < c->np; ++p) plist[pfill[pscene[p]]++] = p;
        std::vector<float4> planes(c->np);
        for (int p = 0; p < c->np; ++p)
            planes[p] = make_float4(d->planes[4 * p], d->planes[4 * p + 1], d->planes[4 * p + 2], d->planes[4 * p + 3]);
        // joints
        std::vector<int2> jab(c->nj);
        std::vector<float4> janc(2 * (size_t)c->nj);
        std::vector<int> jscene(c->nj, 0);
        for (int j = 0; j < c->nj; ++j) {
            int a = d->joint_bodies[2 * j], b = d->joint_bodies[2 * j + 1];
            if (a < -1 || a >= n || b < -1 || b >= n || (a < 0 && b < 0))
                return fail(c, OVL_ERR_ARG, "scene: joint bodies out of range");
            if (a >= 0 && b >= 0 && sob[a] != sob[b]) return fail(c, OVL_ERR_ARG, "scene: joint across scenes");
            jab[j] = make_int2(a, b);
            const float *an = d->joint_anchors + 6 * (size_t)j;
            janc[2 * j] = make_float4(an[0], an[1], an[2], 0.f);
            janc[2 * j + 1] = make_float4(an[3], an[4], an[5], 0.f);
            jscene[j] = a >= 0 ? sob[a] : sob[b];
        }
        // largest contact distance sets the grid cell
        float rmax = 0.f;
        for (int b = 0; b < n; ++b) rmax = std::max(rmax, d->radius[b]);
        c->cs = (2.f * rmax + c->P.margin) * 1.01f;
        // Neighbour capacity per body.  Spheres that touch body a (centres
        // within r_a + r_b + margin) and barely overlap one another are seen
        // from a's centre under disjoint cones of half-angle at least
        // asin(r_min / (r_a + r_min + margin)), so at most
        // 2 / (1 - cos(theta)) of them fit around it; 25 % slack covers the
        // small penetrations the solver leaves.  Never below OVL_MAX_NEIGH.
        {
            std::vector<float> rmin(ns, INFINITY);
            for (int b = 0; b < n; ++b) rmin[sob[b]] = std::min(rmin[sob[b]], d->radius[b]);
            std::vector<long long> off(n + 1, 0);
            for (int b = 0; b < n; ++b) {
                const double rm = rmin[sob[b]];
                const double sn = rm / ((double)d->radius[b] + rm + (double)c->P.margin);
                const double cap = 1.25 * 2.0 / (1.0 - std::sqrt(std::max(0.0, 1.0 - sn * sn)));
                off[b + 1] = off[b] + std::max<long long>(OVL_MAX_NEIGH, (long long)std::ceil(cap));
            }
            c->nb_total = off[n];
            upload(c->nb_off, off.data(), (size_t)n + 1, s);
        }
        c->tsize = next_pow2(2ull * (uint64_t)n);
        // host scene for the sequential algorithms
        c->hs.n = n; c->hs.ns = ns; c->hs.n_parts = c->n_parts;
        c->hs.inv_mass = c->h_im; c->hs.sob = sob; c->hs.part_base = part_base;
        c->hs.scene_gamma.assign(d->scene_gamma, d->scene_gamma + ns);
        c->hs.n_sets.assign(d->n_sets, d->n_sets + ns);
        c->hs.body_base = c->h_body_base;
        c->hs.jab.assign(d->joint_bodies, d->joint_bodies + 2 * (size_t)c->nj);
        // device copies
        upload(c->radius, d->radius, n, s);
        upload(c->im, d->inv_mass, n, s);
        upload(c->sob, sob.data(), n, s);
        upload(c->scene_mu, d->scene_mu, ns, s);
        upload(c->scene_dt, d->scene_dt, ns, s);
        upload(c->scene_flags, d->scene_flags, ns, s);
        upload(c->scene_beta, d->scene_beta, ns, s);
        upload(c->scene_gamma, d->scene_gamma, ns, s);
        upload(c->n_sets, d->n_sets, ns, s);
        upload(c->part_base, part_base.data(), ns + 1, s);
        upload(c->body_base, c->h_body_base.data(), ns + 1, s);
        upload(c->part_scene, c->h_part_scene.data(), c->n_parts, s);
        upload(c->vb_base, vb.data(), ns + 1, s);
        upload(c->planes, planes.data(), c->np, s);
        upload(c->plane_ptr, c->h_plane_ptr.data(), ns + 1, s);
        upload(c->plane_list, plist.data(), c->np, s);
        upload(c->jab, jab.data(), c->nj, s);
        upload(c->janc, janc.data(), 2 * (size_t)c->nj, s);
        upload(c->joint_scene, jscene.data(), c->nj, s);
        // state
        DBuf<float> tmp13;
        upload(tmp13, d->state, 13 * (size_t)n, s);
        c->st.ensure(4 * (size_t)n);
        c->st_alt.ensure(4 * (size_t)n);
        launch_pack_state(tmp13.p, c->radius.p, c->im.p, n, c->st.p, s);
        CK(cudaStreamSynchronize(s));
        tmp13.release();
        c->mask.ensure(n);
        CK(cudaMemsetAsync(c->mask.p, 0, sizeof(uint64_t) * n, s));
        reset_warmstart(c);
        CK(cudaMemsetAsync(c->status.p, 0, 4 * sizeof(int), s));
        CK(cudaStreamSynchronize(s));
        // boxes: half extents and the body-frame inverse inertia of a solid box,
        // 1/I_k = 3 (1/m) / (h_j^2 + h_l^2)
        c->has_boxes = boxes;
        c->h_half.assign(3 * (size_t)n, 0.f);
        if (boxes) {
            std::copy(d->half_extents, d->half_extents + 3 * (size_t)n, c->h_half.begin());
            std::vector<float4> hv(n), iv(n);
            for (int b = 0; b < n; ++b) {
                const float *h = d->half_extents + 3 * (size_t)b;
                const float im = d->inv_mass[b];
                hv[b] = make_float4(h[0], h[1], h[2], 0.f);
                float i3[3] = {0.f, 0.f, 0.f};
                if (h[0] > 0.f || h[1] > 0.f || h[2] > 0.f)
                    for (int k = 0; k < 3; ++k) {
                        const float a = h[(k + 1) % 3], e = h[(k + 2) % 3];
                        i3[k] = im > 0.f ? 3.f * im / (a * a + e * e) : 0.f;
                    }
                iv[b] = make_float4(i3[0], i3[1], i3[2], 0.f);
            }
            upload(c->half, hv.data(), (size_t)n, s);
            upload(c->iib, iv.data(), (size_t)n, s);
            CK(cudaStreamSynchronize(s));
        }
        c->step_index = 0;
        c->have_step = false;
        c->has_scene = true;
        return OVL_OK;
    });
}

ovl_status ovl_set_partition(ovl_ctx *c, const int32_t *set_of_body) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !set_of_body) return fail(c, OVL_ERR_ARG, "no scene or null partition");
        std::vector<uint64_t> m(c->n, 0);
        for (int b = 0; b < c->n; ++b) {
            if (!(c->h_im[b] > 0.f)) continue;
            int w = set_of_body[b];
            if (w < 0 || w >= c->hs.n_sets[c->hs.sob[b]])
                return fail(c, OVL_ERR_MEMBERSHIP, "partition: worker index out of range for body " + std::to_string(b));
            m[b] = 1ull << w;
        }
        upload_masks(c, m);
        return OVL_OK;
    });
}

ovl_status ovl_set_membership(ovl_ctx *c, const uint64_t *masks) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !masks) return fail(c, OVL_ERR_ARG, "no scene or null masks");
        try {
            validate_masks(c, masks);
        } catch (const std::invalid_argument &e) {
            return fail(c, OVL_ERR_MEMBERSHIP, e.what());
        }
        upload_masks(c, std::vector<uint64_t>(masks, masks + c->n));
        return OVL_OK;
    });
}

ovl_status ovl_read_membership(ovl_ctx *c, uint64_t *masks) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !masks) return fail(c, OVL_ERR_ARG, "no scene or null output");
        std::vector<uint64_t> m = download_masks(c);
        std::copy(m.begin(), m.end(), masks);
        return OVL_OK;
    });
}

ovl_status ovl_assign_overlap(ovl_ctx *c) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene) return fail(c, OVL_ERR_ARG, "no scene");
        std::vector<uint64_t> m = download_masks(c);
        try {
            validate_masks(c, m.data());
        } catch (const std::invalid_argument &e) {
            return fail(c, OVL_ERR_MEMBERSHIP, e.what());
        }
        host_assign_overlap(c->hs, m);
        upload_masks(c, m);
        return OVL_OK;
    });
}

ovl_status ovl_set_state(ovl_ctx *c, const float *state13, int32_t on_device) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !state13) return fail(c, OVL_ERR_ARG, "no scene or null state");
        const float *src = state13;
        if (!on_device) {
            upload(c->stage13, state13, 13 * (size_t)c->n, c->stream);
            src = c->stage13.p;
        }
        launch_pack_state(src, c->radius.p, c->im.p, c->n, c->st.p, c->stream);
        if (!on_device) CK(cudaStreamSynchronize(c->stream));   // the host array may be reused
        return OVL_OK;
    });
}

ovl_status ovl_read_state(ovl_ctx *c, float *state13, int32_t on_device) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !state13) return fail(c, OVL_ERR_ARG, "no scene or null output");
        if (on_device) {
            launch_unpack_state(c->st.p, c->n, state13, c->stream);
            return OVL_OK;
        }
        c->stage13.ensure(13 * (size_t)c->n);
        launch_unpack_state(c->st.p, c->n, c->stage13.p, c->stream);
        download(state13, c->stage13.p, 13 * (size_t)c->n, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return OVL_OK;
    });
}

ovl_status ovl_joint_error(ovl_ctx *c, double *sum, double *max_gap) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene) return fail(c, OVL_ERR_ARG, "no scene");
        double h[2] = {0.0, 0.0};
        if (c->nj > 0) {
            c->jerr.ensure(2);
            launch_joint_error(c->jab.p, c->janc.p, c->st.p, c->nj, c->jerr.p, c->stream);
            download(h, c->jerr.p, 2, c->stream);
            CK(cudaStreamSynchronize(c->stream));
        }
        if (sum) *sum = h[0];
        if (max_gap) *max_gap = h[1];
        return OVL_OK;
    });
}

ovl_status ovl_set_step_index(ovl_ctx *c, int64_t k) {
    if (!c) return OVL_ERR_ARG;
    if (k < 0) return fail(c, OVL_ERR_ARG, "step index must be >= 0");
    c->step_index = k;
    return OVL_OK;
}

ovl_status ovl_set_warmstart(ovl_ctx *c, int64_t n, const int32_t *part, const uint64_t *key,
                             const float *lambda3) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || n < 0 || (n > 0 && (!part || !key || !lambda3)))
            return fail(c, OVL_ERR_ARG, "warm start: bad arguments");
        std::vector<int64_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        for (int64_t i = 0; i < n; ++i)
            if (part[i] < 0 || part[i] >= c->n_parts) return fail(c, OVL_ERR_ARG, "warm start: worker out of range");
        std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
            return part[x] != part[y] ? part[x] < part[y] : key[x] < key[y];
        });
        std::vector<int> pstart(c->n_parts + 1, 0);
        std::vector<uint64_t> k(n);
        std::vector<float4> l(n);
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = order[i];
            pstart[part[o] + 1]++;
            k[i] = key[o];
            l[i] = make_float4(lambda3[3 * o], lambda3[3 * o + 1], lambda3[3 * o + 2], 0.f);
        }
        for (int p = 0; p < c->n_parts; ++p) pstart[p + 1] += pstart[p];
        upload(c->ws_pstart, pstart.data(), pstart.size(), c->stream);
        upload(c->ws_key, k.data(), (size_t)n, c->stream);
        upload(c->ws_lam, l.data(), (size_t)n, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        c->ws_n = n;
        return OVL_OK;
    });
}

ovl_status ovl_read_warmstart(ovl_ctx *c, int64_t cap, int64_t *n, int32_t *part, uint64_t *key,
                              float *lambda3) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !n) return fail(c, OVL_ERR_ARG, "no scene or null count");
        *n = c->ws_n;
        if (cap <= 0) return OVL_OK;
        int64_t m = std::min(cap, c->ws_n);
        std::vector<int> pstart(c->n_parts + 1);
        std::vector<float4> l(m);
        download(pstart.data(), c->ws_pstart.p, pstart.size(), c->stream);
        if (key) download(key, c->ws_key.p, (size_t)m, c->stream);
        download(l.data(), c->ws_lam.p, (size_t)m, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        for (int p = 0; p < c->n_parts; ++p)
            for (int64_t i = pstart[p]; i < pstart[p + 1] && i < m; ++i)
                if (part) part[i] = p;
        if (lambda3)
            for (int64_t i = 0; i < m; ++i) {
                lambda3[3 * i] = l[i].x; lambda3[3 * i + 1] = l[i].y; lambda3[3 * i + 2] = l[i].z;
            }
        return OVL_OK;
    });
}

ovl_status ovl_step(ovl_ctx *c, float dt, int32_t iters) {
    return guarded(c, [&]() -> ovl_status { return run_step(c, dt, iters); });
}

ovl_status ovl_step_n(ovl_ctx *c, float dt, int32_t iters, int32_t nsteps, int32_t *done) {
    return guarded(c, [&]() -> ovl_status {
        if (done) *done = 0;
        if (nsteps < 0) return fail(c, OVL_ERR_ARG, "nsteps must be >= 0");
        for (int32_t k = 0; k < nsteps; ++k) {
            const ovl_status rc = run_step(c, dt, iters);
            if (rc != OVL_OK) return rc;
            if (done) *done = k + 1;
        }
        return OVL_OK;
    });
}

ovl_status ovl_load_balance(ovl_ctx *c, int32_t flags) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene) return fail(c, OVL_ERR_ARG, "no scene");
        phase_contacts(c);
        phase_graph(c);
        phase_load_balance(c, (flags & 1) != 0, (flags & 2) != 0);
        return check_device_status(c);
    });
}

ovl_status ovl_sync(ovl_ctx *c) {
    return guarded(c, [&]() -> ovl_status {
        CK(cudaStreamSynchronize(c->stream));
        return OVL_OK;
    });
}

ovl_status ovl_read_stats(ovl_ctx *c, ovl_stats *out) {
    return guarded(c, [&]() -> ovl_status {
        if (!out) return fail(c, OVL_ERR_ARG, "null output");
        std::memset(out, 0, sizeof(*out));
        out->n_workers = c->n_parts;
        if (!c->have_step) return OVL_OK;
        out->n_contacts = c->nc;
        out->n_adjacency = c->nadj;
        out->n_entries = c->ne;
        out->n_pairs = c->npairs;
        out->n_rows = 3ll * c->npairs;
        std::vector<int> ep(c->n + 1), ncol(c->n_parts), its(c->n_parts), rounds(c->n_parts);
        download(rounds.data(), c->part_rounds.p, rounds.size(), c->stream);
        std::vector<double> rs(c->n_parts);
        download(ep.data(), c->entry_ptr.p, ep.size(), c->stream);
        download(ncol.data(), c->part_ncol.p, ncol.size(), c->stream);
        download(its.data(), c->part_iters.p, its.size(), c->stream);
        download(rs.data(), c->part_res_sq.p, rs.size(), c->stream);
        int dstat = 0;
        download(&dstat, c->status.p, 1, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        for (int b = 0; b < c->n; ++b) out->n_overlap += (ep[b + 1] - ep[b]) >= 2;
        double sq = 0;
        for (int p = 0; p < c->n_parts; ++p) {
            out->max_colours = std::max(out->max_colours, ncol[p]);
            out->max_iters = std::max(out->max_iters, its[p]);
            out->colour_rounds_max = std::max(out->colour_rounds_max, rounds[p]);
            sq += rs[p];
        }
        out->residual_rms = c->npairs > 0 ? std::sqrt(sq / (3.0 * c->npairs)) : 0.0;
        out->device_status = dstat;
        for (int i = 0; i < 11; ++i) out->phase_ms[i] = c->phase_ms[i];
        out->n_launches = c->last_launches;
        out->solve_cluster = c->last_cluster;
        out->solve_threads = c->last_threads;
        out->solve_rows_per_thread = c->last_unroll;
        out->solve_ctas = c->last_ctas;
        out->solve_ctas_masses = c->last_ctas_masses;
        out->lb_candidates = c->lb_candidates;
        out->lb_host_ms = c->lb_host_ms;
        return OVL_OK;
    });
}

ovl_status ovl_read_contact_points(ovl_ctx *c, int32_t *k, float *point) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        std::vector<float4> h_p(c->nc, make_float4(0.f, 0.f, 0.f, 0.f));
        if (c->has_boxes) download(h_p.data(), c->c_p.p, c->nc, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < c->nc; ++i) {
            int32_t kk = 0;
            std::memcpy(&kk, &h_p[i].w, sizeof kk);   // stored as the float's bits
            if (k) k[i] = c->has_boxes ? kk : 0;
            if (point) { point[3 * i] = h_p[i].x; point[3 * i + 1] = h_p[i].y; point[3 * i + 2] = h_p[i].z; }
        }
        return OVL_OK;
    });
}

ovl_status ovl_read_contacts(ovl_ctx *c, int32_t *ab, float *phi, float *normal, float *t1) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        std::vector<int2> h_ab(c->nc);
        std::vector<float4> h_n(c->nc), h_t(c->nc);
        download(h_ab.data(), c->c_ab.p, c->nc, c->stream);
        download(h_n.data(), c->c_n.p, c->nc, c->stream);
        download(h_t.data(), c->c_t1.p, c->nc, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < c->nc; ++i) {
            if (ab) { ab[2 * i] = h_ab[i].x; ab[2 * i + 1] = h_ab[i].y; }
            if (phi) phi[i] = h_n[i].w;
            if (normal) { normal[3 * i] = h_n[i].x; normal[3 * i + 1] = h_n[i].y; normal[3 * i + 2] = h_n[i].z; }
            if (t1) { t1[3 * i] = h_t[i].x; t1[3 * i + 1] = h_t[i].y; t1[3 * i + 2] = h_t[i].z; }
        }
        return OVL_OK;
    });
}

ovl_status ovl_read_graph(ovl_ctx *c, int32_t *row_ptr, int32_t *col) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        if (row_ptr) download(row_ptr, c->row_ptr.p, (size_t)c->n + 1, c->stream);
        if (col) download(col, c->col.p, (size_t)c->nadj, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return OVL_OK;
    });
}

ovl_status ovl_read_entries(ovl_ctx *c, int32_t *entry_ptr, int32_t *part, uint8_t *D, float *weight,
                            float *copies13) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        if (entry_ptr) download(entry_ptr, c->entry_ptr.p, (size_t)c->n + 1, c->stream);
        if (part) download(part, c->entry_part.p, (size_t)c->ne, c->stream);
        if (D) download(D, c->D.p, (size_t)c->ne, c->stream);
        if (weight) download(weight, c->weight.p, (size_t)c->ne, c->stream);
        std::vector<float4> cp;
        if (copies13) {
            cp.resize(4 * (size_t)c->ne);
            download(cp.data(), c->copies.p, cp.size(), c->stream);
        }
        CK(cudaStreamSynchronize(c->stream));
        if (copies13)
            for (int e = 0; e < c->ne; ++e) {
                float *o = copies13 + 13 * (size_t)e;
                const float4 x = cp[4 * e], q = cp[4 * e + 1], v = cp[4 * e + 2], w = cp[4 * e + 3];
                o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = q.x; o[4] = q.y; o[5] = q.z; o[6] = q.w;
                o[7] = v.x; o[8] = v.y; o[9] = v.z; o[10] = w.x; o[11] = w.y; o[12] = w.z;
            }
        return OVL_OK;
    });
}

ovl_status ovl_read_pairs(ovl_ctx *c, int32_t *part, uint64_t *key, int32_t *colour, float *lambda3) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        // after the step the pair keys and impulses are the warm-start cache
        if (part) download(part, c->ps_part.p, (size_t)c->npairs, c->stream);
        if (key) download(key, c->ws_key.p, (size_t)c->npairs, c->stream);
        if (colour) download(colour, c->p_colour.p, (size_t)c->npairs, c->stream);
        std::vector<float4> l;
        if (lambda3) {
            l.resize(c->npairs);
            download(l.data(), c->ws_lam.p, (size_t)c->npairs, c->stream);
        }
        CK(cudaStreamSynchronize(c->stream));
        if (lambda3)
            for (int i = 0; i < c->npairs; ++i) {
                lambda3[3 * i] = l[i].x; lambda3[3 * i + 1] = l[i].y; lambda3[3 * i + 2] = l[i].z;
            }
        return OVL_OK;
    });
}

ovl_status ovl_read_worker_stats(ovl_ctx *c, int32_t *iters, double *res_sq, int64_t *rows,
                                 int32_t *colours) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        std::vector<int> ps(c->n_parts + 1);
        if (iters) download(iters, c->part_iters.p, (size_t)c->n_parts, c->stream);
        if (res_sq) download(res_sq, c->part_res_sq.p, (size_t)c->n_parts, c->stream);
        if (colours) download(colours, c->part_ncol.p, (size_t)c->n_parts, c->stream);
        download(ps.data(), c->ws_pstart.p, ps.size(), c->stream);
        CK(cudaStreamSynchronize(c->stream));
        if (rows)
            for (int p = 0; p < c->n_parts; ++p) rows[p] = 3ll * (ps[p + 1] - ps[p]);
        return OVL_OK;
    });
}

ovl_status ovl_read_solve_plan(ovl_ctx *c, int32_t *ctas) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step) return fail(c, OVL_ERR_ARG, "no step has run");
        if (!ctas) return fail(c, OVL_ERR_ARG, "ctas is required");
        for (int p = 0; p < c->n_parts; ++p)
            ctas[p] = c->last_plan_per_worker ? c->h_class_C[p] : c->last_cluster;
        return OVL_OK;
    });
}

}  // extern "C"

extern "C" {

ovl_status ovl_autotune_export(ovl_ctx *c, char *buf, size_t cap, size_t *len) {
    return guarded(c, [&]() -> ovl_status {
        std::ostringstream o;
        o << "{";
        bool first = true;
        for (const auto &kv : c->tuned) {
            if (!first) o << ", ";
            first = false;
            o << "\"" << kv.first << "\": {\"cluster\": " << kv.second.cluster << ", \"threads\": "
              << kv.second.threads << ", \"rows_per_thread\": " << kv.second.unroll << ", \"per_worker\": "
              << kv.second.shape << ", \"ms\": " << kv.second.ms << "}";
        }
        o << "}";
        std::string t = o.str();
        if (len) *len = t.size();
        if (buf && cap > 0) {
            size_t m = std::min(cap - 1, t.size());
            std::memcpy(buf, t.data(), m);
            buf[m] = 0;
        }
        return OVL_OK;
    });
}

ovl_status ovl_autotune_import(ovl_ctx *c, const char *json) {
    return guarded(c, [&]() -> ovl_status {
        if (!json) return fail(c, OVL_ERR_ARG, "null json");
        // flat format written by ovl_autotune_export
        std::string t(json);
        size_t pos = 0;
        auto num = [&](const std::string &field, size_t from, size_t to) -> double {
            size_t f = t.find("\"" + field + "\"", from);
            if (f == std::string::npos || f > to) throw std::invalid_argument("autotune json: missing " + field);
            f = t.find(':', f);
            return std::strtod(t.c_str() + f + 1, nullptr);
        };
        while ((pos = t.find('"', pos)) != std::string::npos) {
            size_t e = t.find('"', pos + 1);
            if (e == std::string::npos) break;
            std::string key = t.substr(pos + 1, e - pos - 1);
            size_t ob = t.find('{', e), cb = t.find('}', e);
            if (ob == std::string::npos || cb == std::string::npos) break;
            ovl_ctx::TuneCfg cfg;
            cfg.cluster = (int)num("cluster", ob, cb);
            cfg.threads = (int)num("threads", ob, cb);
            cfg.unroll = (int)num("rows_per_thread", ob, cb);
            cfg.ms = (float)num("ms", ob, cb);
            cfg.shape = t.find("\"per_worker\"", ob) < cb ? (int)num("per_worker", ob, cb) : 0;
            bool ok = cfg.shape > 0 ? cfg.shape <= 3
                                    : (cfg.cluster == 1 || cfg.cluster == 2 || cfg.cluster == 4 || cfg.cluster == 8) &&
                                          (cfg.threads >= 32 && cfg.threads <= 512) && (cfg.unroll == 1 || cfg.unroll == 2);
            if (!ok) return fail(c, OVL_ERR_ARG, "autotune json: bad entry " + key);
            c->tuned[key] = cfg;
            pos = cb + 1;
        }
        return OVL_OK;
    });
}

}  // extern "C"
