// mlp.cu -- host side of the learned warm start: the phases a step runs
// (features and the network's proposal before the rows; the log after the
// solve) and the C ABI that sets, trains and evaluates the network.
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"

namespace ovl {

namespace {

constexpr long long kMaxBatch = 1 << 20;
constexpr int kLossChunk = 1 << 16;

bool features_needed(const ovl_ctx *c) {
    return c->ws_mode != OVL_WS_PREVIOUS || c->log_on || (c->P.flags & OVL_FLAG_FEATURES);
}

void ensure_train_buffers(ovl_ctx *c, int batch) {
    c->train_act.ensure((size_t)batch * MLP_ACT_STRIDE);
    c->train_sample_loss.ensure((size_t)batch);
    c->train_partials.ensure((size_t)train_wgrad_blocks(batch) * (MLP_N_PARAMS + 1));
    c->mlp_grad.ensure(MLP_N_PARAMS);
    c->mlp_loss.ensure(1);
}

TrainArgs train_args(ovl_ctx *c, long long first, long long count, int batch, int sampling,
                     uint64_t seed, long long step, int backward) {
    TrainArgs a{};
    a.log_feat = c->log_feat.p; a.log_targ = c->log_targ.p;
    a.first = first; a.count = count; a.batch = batch; a.sampling = sampling;
    a.seed = seed; a.step = step; a.backward = backward;
    a.theta = c->mlp_theta.p;
    a.act = c->train_act.p; a.sample_loss = c->train_sample_loss.p;
    a.partials = c->train_partials.p;
    a.status = c->status.p;
    return a;
}

void check_log_range(const ovl_ctx *c, long long first, long long count) {
    if (first < 0 || count < 1 || first + count > c->log_n)
        throw std::invalid_argument("log rows [" + std::to_string(first) + ", " +
                                    std::to_string(first + count) + ") are outside the " +
                                    std::to_string(c->log_n) + " logged rows");
}

}  // namespace

void phase_warmstart(ovl_ctx *c, float dt_override) {
    c->feat_valid = false;
    if (!features_needed(c)) return;
    if (c->ws_mode != OVL_WS_PREVIOUS && !c->mlp_ready)
        throw std::invalid_argument("the MLP warm start needs the network's parameters (ovl_mlp_set_params)");
    cudaStream_t s = c->stream;
    const int np = c->npairs;
    if (c->P.flags & OVL_FLAG_TIMING) CK(cudaEventRecord(c->ev[12], s));
    c->depth.ensure((size_t)c->n + 1);
    launch_depth(c->mask.p, c->row_ptr.p, c->col.p, c->n, c->depth.p, s);
    c->feat.ensure(4 * (size_t)np + 4);
    c->is_contact.ensure((size_t)np + 1);
    FeatArgs a{};
    a.np = np; a.nc = c->nc; a.n = c->n;
    a.ps_cons = c->ps_cons.p; a.ps_part = c->ps_part.p; a.part_scene = c->part_scene.p;
    a.c_ab = c->c_ab.p; a.c_n = c->c_n.p; a.c_t1 = c->c_t1.p; a.st = c->st.p;
    a.row_ptr = c->row_ptr.p; a.depth = c->depth.p;
    a.scene_dt = c->scene_dt.p; a.scene_mu = c->scene_mu.p; a.dt_override = dt_override;
    const float *g = c->P.gravity;
    a.g_ref = std::fmax(std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]), 1.0f);
    a.p_key = c->p_key.p;
    a.ws.ws_pstart = c->ws_pstart.p; a.ws.ws_key = c->ws_key.p; a.ws.ws_lam = c->ws_lam.p;
    a.ws.factor = c->P.warmstart;
    a.feat = c->feat.p; a.is_contact = c->is_contact.p;
    launch_features(a, s);
    if (c->ws_mode != OVL_WS_PREVIOUS)
        launch_mlp_infer(c->mlp_packed.p, c->feat.p, np, c->ws_mode, c->p_lam0.p, nullptr, 0, c->status.p, s);
    if (c->P.flags & OVL_FLAG_TIMING) CK(cudaEventRecord(c->ev[13], s));
    c->feat_valid = true;
}

void phase_log(ovl_ctx *c) {
    if (!c->log_on || !c->feat_valid || c->log_n >= c->log_cap || c->npairs == 0) return;
    const int np = c->npairs;
    c->contact_pos.ensure((size_t)np + 1);
    scan_i32(c->is_contact.p, c->contact_pos.p, np, c->scan_tmp, c->stream);
    const int total = read_i32(c, c->contact_pos.p + np);
    launch_log_append(c->feat.p, c->lam_out.p, c->contact_pos.p, np, c->log_feat.p, c->log_targ.p,
                      c->log_n, c->log_cap, c->stream);
    c->log_n = std::min(c->log_cap, c->log_n + (long long)total);
}

void release_mlp(ovl_ctx *c) {
    c->feat.release(); c->is_contact.release(); c->contact_pos.release(); c->depth.release();
    c->mlp_theta.release(); c->mlp_m.release(); c->mlp_v.release(); c->mlp_grad.release();
    c->mlp_loss.release(); c->mlp_packed.release(); c->log_feat.release(); c->log_targ.release();
    c->train_act.release(); c->train_sample_loss.release(); c->train_partials.release();
    c->train_loss_hist.release(); c->infer_y.release(); c->infer_feat.release(); c->loss_acc.release();
    c->train_c12.release(); c->train_step.release();
}

}  // namespace ovl

extern "C" {

ovl_status ovl_set_warmstart_mode(ovl_ctx *c, int32_t mode) {
    return guarded(c, [&]() -> ovl_status {
        if (mode != OVL_WS_PREVIOUS && mode != OVL_WS_MLP && mode != OVL_WS_MLP_NEW)
            return fail(c, OVL_ERR_ARG, "unknown warm-start mode");
        if (mode != OVL_WS_PREVIOUS && !c->mlp_ready)
            return fail(c, OVL_ERR_ARG, "set the network's parameters (ovl_mlp_set_params) first");
        c->ws_mode = mode;
        return OVL_OK;
    });
}

ovl_status ovl_read_features(ovl_ctx *c, float *feat12, float *scale, int32_t *found,
                             float *lambda0_3) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->have_step || !c->feat_valid)
            return fail(c, OVL_ERR_ARG, "the last step computed no features");
        const size_t np = (size_t)c->npairs;
        std::vector<float4> f(4 * np + 1), l(np + 1);
        download(f.data(), c->feat.p, 4 * np, c->stream);
        download(l.data(), c->p_lam0.p, np, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        for (size_t k = 0; k < np; ++k) {
            const float *r = reinterpret_cast<const float *>(&f[4 * k]);
            if (feat12) std::memcpy(feat12 + 12 * k, r, 12 * sizeof(float));
            if (scale) scale[k] = r[13];
            if (found) found[k] = r[12] != 0.f;
            if (lambda0_3) { lambda0_3[3 * k] = l[k].x; lambda0_3[3 * k + 1] = l[k].y; lambda0_3[3 * k + 2] = l[k].z; }
        }
        return OVL_OK;
    });
}

ovl_status ovl_mlp_set_params(ovl_ctx *c, const float *theta, int32_t n) {
    return guarded(c, [&]() -> ovl_status {
        if (!theta || n != MLP_N_PARAMS) return fail(c, OVL_ERR_ARG, "expected OVL_MLP_N_PARAMS parameters");
        for (int i = 0; i < n; ++i)
            if (!std::isfinite(theta[i])) return fail(c, OVL_ERR_NONFINITE, "non-finite parameter");
        upload(c->mlp_theta, theta, (size_t)n, c->stream);
        c->mlp_m.ensure(n); c->mlp_v.ensure(n);
        CK(cudaMemsetAsync(c->mlp_m.p, 0, sizeof(float) * n, c->stream));
        CK(cudaMemsetAsync(c->mlp_v.p, 0, sizeof(float) * n, c->stream));
        c->mlp_packed.ensure(MLP_PK_WORDS);
        launch_mlp_pack(c->mlp_theta.p, c->mlp_packed.p, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        c->adam_t = 0;
        c->mlp_ready = true;
        return OVL_OK;
    });
}

ovl_status ovl_mlp_get_params(ovl_ctx *c, float *theta, int32_t n) {
    return guarded(c, [&]() -> ovl_status {
        if (!theta || n != MLP_N_PARAMS) return fail(c, OVL_ERR_ARG, "expected OVL_MLP_N_PARAMS parameters");
        if (!c->mlp_ready) return fail(c, OVL_ERR_ARG, "no parameters set");
        download(theta, c->mlp_theta.p, (size_t)n, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return OVL_OK;
    });
}

ovl_status ovl_mlp_forward(ovl_ctx *c, int64_t n, const float *feat12, float *y3) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->mlp_ready) return fail(c, OVL_ERR_ARG, "no parameters set");
        if (n < 0 || n > (int64_t)1 << 30 || (n > 0 && (!feat12 || !y3)))
            return fail(c, OVL_ERR_ARG, "bad size or null array");
        if (n == 0) return OVL_OK;
        std::vector<float> rows(16 * (size_t)n, 0.f);
        for (int64_t k = 0; k < n; ++k) std::memcpy(&rows[16 * k], feat12 + 12 * k, 12 * sizeof(float));
        c->infer_feat.ensure(4 * (size_t)n);
        CK(cudaMemcpyAsync(c->infer_feat.p, rows.data(), rows.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        c->infer_y.ensure(3 * (size_t)n);
        launch_mlp_infer(c->mlp_packed.p, c->infer_feat.p, (int)n, 0, nullptr, c->infer_y.p, 0, c->status.p, c->stream);
        download(y3, c->infer_y.p, 3 * (size_t)n, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return check_device_status(c);
    });
}

ovl_status ovl_log_reserve(ovl_ctx *c, int64_t capacity) {
    return guarded(c, [&]() -> ovl_status {
        if (capacity < 0) return fail(c, OVL_ERR_ARG, "negative capacity");
        c->log_feat.release(); c->log_targ.release();
        c->log_n = 0; c->log_cap = 0; c->log_on = false;
        if (capacity > 0) {
            c->log_feat.ensure(12 * (size_t)capacity);
            c->log_targ.ensure(3 * (size_t)capacity);
            c->log_cap = capacity;
        }
        return OVL_OK;
    });
}

ovl_status ovl_log_enable(ovl_ctx *c, int32_t on) {
    return guarded(c, [&]() -> ovl_status {
        if (on && c->log_cap == 0) return fail(c, OVL_ERR_ARG, "reserve the log first");
        c->log_on = on != 0;
        return OVL_OK;
    });
}

ovl_status ovl_log_size(ovl_ctx *c, int64_t *n) {
    return guarded(c, [&]() -> ovl_status {
        if (!n) return fail(c, OVL_ERR_ARG, "null output");
        *n = c->log_n;
        return OVL_OK;
    });
}

ovl_status ovl_log_append(ovl_ctx *c, int64_t n, const float *feat12, const float *target3) {
    return guarded(c, [&]() -> ovl_status {
        if (n < 0 || (n > 0 && (!feat12 || !target3))) return fail(c, OVL_ERR_ARG, "bad size or null array");
        if (c->log_n + n > c->log_cap) return fail(c, OVL_ERR_CAPACITY, "the log is full");
        if (n == 0) return OVL_OK;
        CK(cudaMemcpyAsync(c->log_feat.p + 12 * c->log_n, feat12, 12 * sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->log_targ.p + 3 * c->log_n, target3, 3 * sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->log_n += n;
        return OVL_OK;
    });
}

ovl_status ovl_log_read(ovl_ctx *c, int64_t first, int64_t n, float *feat12, float *target3) {
    return guarded(c, [&]() -> ovl_status {
        if (n == 0) return OVL_OK;
        check_log_range(c, first, n);
        if (feat12) download(feat12, c->log_feat.p + 12 * first, 12 * (size_t)n, c->stream);
        if (target3) download(target3, c->log_targ.p + 3 * first, 3 * (size_t)n, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return OVL_OK;
    });
}

ovl_status ovl_mlp_train(ovl_ctx *c, const ovl_train_desc *d, float *loss_per_step) {
    return guarded(c, [&]() -> ovl_status {
        if (!d) return fail(c, OVL_ERR_ARG, "null descriptor");
        if (!c->mlp_ready) return fail(c, OVL_ERR_ARG, "no parameters set");
        check_log_range(c, d->first, d->count);
        if (d->batch < 1 || d->batch > kMaxBatch) return fail(c, OVL_ERR_ARG, "batch must be in [1, 1048576]");
        if (d->steps < 0 || (d->sampling != 0 && d->sampling != 1)) return fail(c, OVL_ERR_ARG, "bad steps or sampling");
        const float lr = d->lr > 0.f ? d->lr : 1e-3f;
        const float b1 = d->beta1 > 0.f ? d->beta1 : 0.9f, b2 = d->beta2 > 0.f ? d->beta2 : 0.999f;
        const float eps = d->eps > 0.f ? d->eps : 1e-8f;
        if (b1 >= 1.f || b2 >= 1.f) return fail(c, OVL_ERR_ARG, "Adam betas must be below 1");
        ensure_train_buffers(c, d->batch);
        const int steps = d->steps;
        c->train_loss_hist.ensure((size_t)steps + 1);
        // Adam's bias corrections of every step of the call, and the step
        // counter, live in device memory, so every step launches the same
        // kernels with the same arguments: a block of steps is captured once
        // as a CUDA graph and replayed
        std::vector<float> c12(2 * (size_t)steps + 2);
        for (int t = 0; t < steps; ++t) {
            const double k = (double)(c->adam_t + 1 + t);
            c12[2 * t] = (float)(1.0 / (1.0 - std::pow((double)b1, k)));
            c12[2 * t + 1] = (float)(1.0 / (1.0 - std::pow((double)b2, k)));
        }
        upload(c->train_c12, c12.data(), c12.size(), c->stream);
        c->train_step.ensure(1);
        CK(cudaMemsetAsync(c->train_step.p, 0, sizeof(long long), c->stream));
        const int blocks = train_wgrad_blocks(d->batch);
        TrainArgs a = train_args(c, d->first, d->count, d->batch, d->sampling, d->seed, 0, 1);
        a.step_dev = c->train_step.p;
        auto one_step = [&](cudaStream_t st) {
            launch_train_fwd(a, st);
            launch_train_wgrad(a, st);
            launch_train_reduce_dev(c->train_partials.p, blocks, d->batch, c->train_loss_hist.p,
                                    c->mlp_theta.p, c->mlp_m.p, c->mlp_v.p, lr, b1, b2, eps,
                                    c->train_c12.p, c->train_step.p, st);
        };
        constexpr int kGraphSteps = 50;
        int done = 0;
        if (steps >= 2 * kGraphSteps) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            try {
                for (int t = 0; t < kGraphSteps; ++t) one_step(c->stream);
            } catch (...) {
                cudaGraph_t partial = nullptr;
                cudaStreamEndCapture(c->stream, &partial);   // leave the stream usable
                if (partial) cudaGraphDestroy(partial);
                throw;
            }
            CK(cudaStreamEndCapture(c->stream, &g));
            cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            CK(e);
            for (; done + kGraphSteps <= steps; done += kGraphSteps) {
                e = cudaGraphLaunch(ge, c->stream);
                if (e != cudaSuccess) break;
            }
            cudaGraphExecDestroy(ge);
            CK(e);
        }
        for (; done < steps; ++done) one_step(c->stream);
        c->adam_t += steps;
        launch_mlp_pack(c->mlp_theta.p, c->mlp_packed.p, c->stream);
        if (loss_per_step && d->steps > 0) download(loss_per_step, c->train_loss_hist.p, (size_t)d->steps, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        return check_device_status(c);
    });
}

ovl_status ovl_mlp_grad(ovl_ctx *c, int64_t first, int64_t count, float *grad, double *loss) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->mlp_ready) return fail(c, OVL_ERR_ARG, "no parameters set");
        check_log_range(c, first, count);
        if (count > kMaxBatch) return fail(c, OVL_ERR_ARG, "count must be <= 1048576");
        const int batch = (int)count;
        ensure_train_buffers(c, batch);
        TrainArgs a = train_args(c, first, count, batch, 0, 0, 0, 1);
        launch_train_fwd(a, c->stream);
        launch_train_wgrad(a, c->stream);
        launch_train_reduce(c->train_partials.p, train_wgrad_blocks(batch), batch, c->mlp_grad.p,
                            c->mlp_loss.p, 0, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f,
                            c->stream);
        float l = 0.f;
        if (grad) download(grad, c->mlp_grad.p, (size_t)MLP_N_PARAMS, c->stream);
        download(&l, c->mlp_loss.p, 1, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        if (loss) *loss = l;
        return check_device_status(c);
    });
}

ovl_status ovl_mlp_loss(ovl_ctx *c, int64_t first, int64_t count, double *loss) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->mlp_ready) return fail(c, OVL_ERR_ARG, "no parameters set");
        if (!loss) return fail(c, OVL_ERR_ARG, "null output");
        check_log_range(c, first, count);
        ensure_train_buffers(c, kLossChunk);
        c->loss_acc.ensure(1);
        CK(cudaMemsetAsync(c->loss_acc.p, 0, sizeof(double), c->stream));
        for (long long off = 0; off < count; off += kLossChunk) {
            const int b = (int)std::min<long long>(kLossChunk, count - off);
            TrainArgs a = train_args(c, first + off, b, b, 0, 0, 0, 0);
            launch_train_fwd(a, c->stream);
            launch_loss_sum(c->train_sample_loss.p, b, c->loss_acc.p, c->stream);
        }
        double acc = 0.0;
        download(&acc, c->loss_acc.p, 1, c->stream);
        CK(cudaStreamSynchronize(c->stream));
        *loss = acc / (3.0 * (double)count);
        return OVL_OK;
    });
}

}  // extern "C"
