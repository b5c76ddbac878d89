// checkpoint.cu -- ovl_save / ovl_load: the state a step reads, as one
// versioned byte blob, so that a run can stop and resume (the paper's
// "get / reset state" of a worker, Table 1, for the whole simulation).
//
// A step of Algorithm 1 reads: the blended body state, every body's worker
// mask W_b, the warm-start cache (previous impulses per (worker, constraint
// key)), the step index (the removal cadence of Algorithm 6) and, with the
// learned warm start, the network's parameters.  The blob holds exactly
// those, plus Adam's moments (training resumes where it stopped) and the
// autotuner's table (launch shapes, which change no bit of a result).  The
// scene itself is not in it: ovl_load expects the same scene uploaded and
// refuses another one (a hash of its host arrays and its sizes).
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "ovl.h"

namespace {

constexpr char kMagic[8] = {'O', 'V', 'L', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

struct SaveHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n, n_parts, ns, ws_mode;
    int64_t step_index, ws_n;
    uint64_t scene_hash;
    int32_t mlp_ready, mlp_params;
    int64_t adam_t, tune_bytes;
};

// FNV-1a over the scene's host arrays
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    template <class T>
    void add(const std::vector<T> &v) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(v.data());
        for (size_t i = 0; i < v.size() * sizeof(T); ++i) { h ^= p[i]; h *= 1099511628211ull; }
        const uint64_t n = v.size();
        for (int i = 0; i < 8; ++i) { h ^= (n >> (8 * i)) & 0xffu; h *= 1099511628211ull; }
    }
};

uint64_t scene_hash(const ovl_ctx *c) {
    Fnv f;
    f.add(c->h_radius);
    f.add(c->hs.inv_mass);
    f.add(c->hs.sob);
    f.add(c->hs.n_sets);
    f.add(c->hs.scene_gamma);
    f.add(c->hs.jab);
    f.add(c->h_plane_ptr);
    f.add(c->h_half);
    return f.h;
}

size_t payload_bytes(const SaveHeader &h) {
    size_t b = 4 * sizeof(float4) * (size_t)h.n + sizeof(uint64_t) * (size_t)h.n;
    b += sizeof(int) * ((size_t)h.n_parts + 1) + (sizeof(uint64_t) + sizeof(float4)) * (size_t)h.ws_n;
    if (h.mlp_ready) b += 3 * sizeof(float) * (size_t)h.mlp_params;
    return b + (size_t)h.tune_bytes;
}

std::string tune_text(ovl_ctx *c) {
    size_t len = 0;
    if (ovl_autotune_export(c, nullptr, 0, &len) != OVL_OK) throw std::runtime_error("autotune export failed");
    std::string t(len + 1, '\0');
    if (ovl_autotune_export(c, &t[0], t.size(), &len) != OVL_OK) throw std::runtime_error("autotune export failed");
    t.resize(len);
    return t;
}

}  // namespace

extern "C" {

ovl_status ovl_save(ovl_ctx *c, void *buf, size_t cap, size_t *len) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !len) return fail(c, OVL_ERR_ARG, "save: no scene or null length");
        SaveHeader h{};
        std::memcpy(h.magic, kMagic, sizeof kMagic);
        h.version = kVersion;
        h.header_bytes = sizeof(SaveHeader);
        h.n = c->n; h.n_parts = c->n_parts; h.ns = c->ns; h.ws_mode = c->ws_mode;
        h.step_index = c->step_index; h.ws_n = c->ws_n;
        h.scene_hash = scene_hash(c);
        h.mlp_ready = c->mlp_ready ? 1 : 0;
        h.mlp_params = OVL_MLP_N_PARAMS;
        h.adam_t = c->adam_t;
        const std::string tune = tune_text(c);
        h.tune_bytes = (int64_t)tune.size();
        *len = sizeof(SaveHeader) + payload_bytes(h);
        if (!buf) return OVL_OK;
        if (cap < *len) return fail(c, OVL_ERR_CAPACITY, "save: buffer smaller than the checkpoint");
        char *p = static_cast<char *>(buf);
        std::memcpy(p, &h, sizeof h);
        p += sizeof h;
        auto take = [&](const void *dev, size_t bytes) {
            if (bytes) CK(cudaMemcpyAsync(p, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
            p += bytes;
        };
        take(c->st.p, 4 * sizeof(float4) * (size_t)c->n);
        take(c->mask.p, sizeof(uint64_t) * (size_t)c->n);
        std::vector<int> pstart(c->n_parts + 1, 0);
        if (c->ws_n > 0 || c->ws_pstart.p) {
            CK(cudaMemcpyAsync(pstart.data(), c->ws_pstart.p, sizeof(int) * pstart.size(), cudaMemcpyDeviceToHost,
                               c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        std::memcpy(p, pstart.data(), sizeof(int) * pstart.size());
        p += sizeof(int) * pstart.size();
        take(c->ws_key.p, sizeof(uint64_t) * (size_t)c->ws_n);
        take(c->ws_lam.p, sizeof(float4) * (size_t)c->ws_n);
        if (h.mlp_ready) {
            take(c->mlp_theta.p, sizeof(float) * OVL_MLP_N_PARAMS);
            take(c->mlp_m.p, sizeof(float) * OVL_MLP_N_PARAMS);
            take(c->mlp_v.p, sizeof(float) * OVL_MLP_N_PARAMS);
        }
        CK(cudaStreamSynchronize(c->stream));
        std::memcpy(p, tune.data(), tune.size());
        return OVL_OK;
    });
}

ovl_status ovl_load(ovl_ctx *c, const void *buf, size_t len) {
    return guarded(c, [&]() -> ovl_status {
        if (!c->has_scene || !buf) return fail(c, OVL_ERR_ARG, "load: no scene or null buffer");
        SaveHeader h;
        if (len < sizeof h) return fail(c, OVL_ERR_ARG, "load: buffer shorter than a checkpoint header");
        std::memcpy(&h, buf, sizeof h);
        if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0 || h.version != kVersion ||
            h.header_bytes != sizeof(SaveHeader))
            return fail(c, OVL_ERR_ARG, "load: not a checkpoint of this library version");
        if (h.n != c->n || h.n_parts != c->n_parts || h.ns != c->ns || h.scene_hash != scene_hash(c))
            return fail(c, OVL_ERR_ARG, "load: the checkpoint belongs to another scene");
        if (h.ws_n < 0 || h.tune_bytes < 0 || h.step_index < 0 || h.mlp_params != OVL_MLP_N_PARAMS ||
            len != sizeof h + payload_bytes(h))
            return fail(c, OVL_ERR_ARG, "load: checkpoint sizes do not add up");
        const char *p = static_cast<const char *>(buf) + sizeof h;
        std::vector<uint64_t> masks(c->n);
        std::memcpy(masks.data(), p + 4 * sizeof(float4) * (size_t)c->n, sizeof(uint64_t) * masks.size());
        for (int b = 0; b < c->n; ++b) {
            const int s = c->hs.sob[b];
            const uint64_t allowed = c->hs.n_sets[s] >= 64 ? ~0ull : ((1ull << c->hs.n_sets[s]) - 1ull);
            if ((masks[b] & ~allowed) || (c->hs.inv_mass[b] > 0.f) != (masks[b] != 0))
                return fail(c, OVL_ERR_MEMBERSHIP, "load: a mask names a worker the scene does not have");
        }
        std::vector<int> pstart(c->n_parts + 1);
        std::memcpy(pstart.data(), p + (4 * sizeof(float4) + sizeof(uint64_t)) * (size_t)c->n,
                    sizeof(int) * pstart.size());
        if (pstart[0] != 0 || pstart[c->n_parts] != h.ws_n)
            return fail(c, OVL_ERR_ARG, "load: warm-start cache offsets are inconsistent");
        for (int q = 0; q < c->n_parts; ++q)
            if (pstart[q + 1] < pstart[q]) return fail(c, OVL_ERR_ARG, "load: warm-start cache offsets decrease");
        auto give = [&](void *dev, size_t bytes) {
            if (bytes) CK(cudaMemcpyAsync(dev, p, bytes, cudaMemcpyHostToDevice, c->stream));
            p += bytes;
        };
        give(c->st.p, 4 * sizeof(float4) * (size_t)c->n);
        give(c->mask.p, sizeof(uint64_t) * (size_t)c->n);
        upload(c->ws_pstart, pstart.data(), pstart.size(), c->stream);
        p += sizeof(int) * pstart.size();
        c->ws_key.ensure((size_t)h.ws_n + 1);
        c->ws_lam.ensure((size_t)h.ws_n + 1);
        give(c->ws_key.p, sizeof(uint64_t) * (size_t)h.ws_n);
        give(c->ws_lam.p, sizeof(float4) * (size_t)h.ws_n);
        if (h.mlp_ready) {
            c->mlp_theta.ensure(OVL_MLP_N_PARAMS); c->mlp_m.ensure(OVL_MLP_N_PARAMS); c->mlp_v.ensure(OVL_MLP_N_PARAMS);
            c->mlp_packed.ensure(MLP_PK_WORDS);
            give(c->mlp_theta.p, sizeof(float) * OVL_MLP_N_PARAMS);
            give(c->mlp_m.p, sizeof(float) * OVL_MLP_N_PARAMS);
            give(c->mlp_v.p, sizeof(float) * OVL_MLP_N_PARAMS);
            launch_mlp_pack(c->mlp_theta.p, c->mlp_packed.p, c->stream);
        }
        CK(cudaStreamSynchronize(c->stream));
        const std::string tune(p, (size_t)h.tune_bytes);
        c->tuned.clear();
        if (!tune.empty()) {
            const ovl_status rc = ovl_autotune_import(c, tune.c_str());
            if (rc != OVL_OK) return rc;
        }
        c->step_index = h.step_index;
        c->ws_n = h.ws_n;
        c->ws_mode = h.ws_mode;
        c->mlp_ready = h.mlp_ready != 0;
        c->adam_t = h.adam_t;
        c->have_step = false;     // the last step's records belong to the run before the load
        c->feat_valid = false;
        return OVL_OK;
    });
}

}  // extern "C"
