// host_api.cpp -- C entry points that run the library's host-side membership
// algorithms (ASSIGNTOOVERLAPSET / GROWOVERLAP, Algorithms 2-3, and
// LOADBALANCE / BRIDGE, Algorithms 6-7, Section 5) on caller-supplied arrays.
// They make no CUDA call, so they run on machines without a GPU; a step runs
// the same functions after reading its contacts back from the device.
#include <stdint.h>

#include <algorithm>
#include <exception>
#include <vector>

#include "common.cuh"
#include "ovl.h"

namespace ovl {
namespace {

// Scenes as contiguous body ranges: scene_of_body non-decreasing, every value
// in [0, n_scenes), 1 <= n_sets <= 64, gamma >= 0.  false on any violation.
bool make_scene(int32_t n, const int32_t *sob, int32_t n_scenes, const int32_t *n_sets,
                const int32_t *scene_gamma, HostScene &sc) {
    if (n < 0 || n_scenes < 1 || (n > 0 && !sob) || !n_sets || !scene_gamma) return false;
    sc.n = n;
    sc.ns = n_scenes;
    sc.sob.assign(sob, sob + n);
    sc.n_sets.assign(n_sets, n_sets + n_scenes);
    sc.scene_gamma.assign(scene_gamma, scene_gamma + n_scenes);
    sc.part_base.assign(n_scenes + 1, 0);
    for (int s = 0; s < n_scenes; ++s) {
        if (n_sets[s] < 1 || n_sets[s] > 64 || scene_gamma[s] < 0) return false;
        sc.part_base[s + 1] = sc.part_base[s] + n_sets[s];
    }
    sc.n_parts = sc.part_base[n_scenes];
    sc.body_base.assign(n_scenes + 1, n);
    for (int b = n - 1; b >= 0; --b) {
        if (sob[b] < 0 || sob[b] >= n_scenes || (b + 1 < n && sob[b] > sob[b + 1])) return false;
        sc.body_base[sob[b]] = b;
    }
    for (int s = n_scenes - 1; s >= 0; --s) sc.body_base[s] = std::min(sc.body_base[s], sc.body_base[s + 1]);
    return true;
}

// every mask bit names a worker of the body's scene
bool masks_valid(const HostScene &sc, const uint64_t *mask) {
    for (int b = 0; b < sc.n; ++b) {
        const int k = sc.n_sets[sc.sob[b]];
        if (k < 64 && (mask[b] >> k) != 0) return false;
    }
    return true;
}

}  // namespace
}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_host_load_balance(int32_t n, const int32_t *scene_of_body, int32_t n_scenes,
                                            const int32_t *n_sets, const int32_t *scene_gamma,
                                            uint64_t *mask, const int32_t *row_ptr, const int32_t *col,
                                            int64_t n_contacts, const int32_t *contact_bodies,
                                            const int32_t *contact_count, int32_t do_activate,
                                            int32_t do_deactivate, int32_t threads) {
    try {
        HostScene sc;
        if (!make_scene(n, scene_of_body, n_scenes, n_sets, scene_gamma, sc)) return OVL_ERR_ARG;
        if (n_contacts < 0 || threads < 1 || threads > 64 || (n > 0 && (!mask || !row_ptr)) ||
            (n_contacts > 0 && !contact_bodies))
            return OVL_ERR_ARG;
        if (!masks_valid(sc, mask)) return OVL_ERR_MEMBERSHIP;
        // graph: CSR over the bodies, edges inside one scene
        if (n > 0 && row_ptr[0] != 0) return OVL_ERR_ARG;
        for (int b = 0; b < n; ++b) {
            if (row_ptr[b + 1] < row_ptr[b]) return OVL_ERR_ARG;
            for (int k = row_ptr[b]; k < row_ptr[b + 1]; ++k)
                if (!col || col[k] < 0 || col[k] >= n || scene_of_body[col[k]] != scene_of_body[b]) return OVL_ERR_ARG;
        }
        // contacts: two bodies of one scene, scenes in ascending order
        std::vector<int2> ab((size_t)n_contacts);
        for (int64_t i = 0; i < n_contacts; ++i) {
            const int a = contact_bodies[2 * i], b = contact_bodies[2 * i + 1];
            if (a < 0 || a >= n || b < 0 || b >= n || scene_of_body[a] != scene_of_body[b]) return OVL_ERR_ARG;
            if (i > 0 && scene_of_body[a] < scene_of_body[ab[i - 1].x]) return OVL_ERR_ARG;
            ab[i] = make_int2(a, b);
        }
        if (contact_count)
            for (int b = 0; b < n; ++b)
                if (contact_count[b] < 0) return OVL_ERR_ARG;
        // live loads <W> of the masks as given (Table 1)
        std::vector<int> loads(sc.n_parts + 1, 0);
        for (int b = 0; b < n; ++b) {
            const int base = sc.part_base[scene_of_body[b]];
            const int w = contact_count ? 1 + contact_count[b] : 1;
            for (uint64_t m = mask[b]; m; m &= m - 1) loads[base + __builtin_ctzll(m)] += w;
        }
        std::vector<BallWorkspace> ws((size_t)threads);
        host_load_balance(sc, mask, loads.data(), contact_count, n_contacts, ab.data(), row_ptr, col,
                          do_activate != 0, do_deactivate != 0, ws);
        return OVL_OK;
    } catch (const std::exception &) {
        return OVL_ERR_ARG;
    }
}

extern "C" ovl_status ovl_host_assign_overlap(int32_t n, const int32_t *scene_of_body, int32_t n_scenes,
                                              const int32_t *n_sets, const int32_t *scene_gamma,
                                              const float *inv_mass, int32_t n_joints,
                                              const int32_t *joint_bodies, uint64_t *mask) {
    try {
        HostScene sc;
        if (!make_scene(n, scene_of_body, n_scenes, n_sets, scene_gamma, sc)) return OVL_ERR_ARG;
        if (n_joints < 0 || (n > 0 && (!mask || !inv_mass)) || (n_joints > 0 && !joint_bodies)) return OVL_ERR_ARG;
        if (!masks_valid(sc, mask)) return OVL_ERR_MEMBERSHIP;
        for (int32_t j = 0; j < 2 * n_joints; ++j)
            if (joint_bodies[j] < -1 || joint_bodies[j] >= n) return OVL_ERR_ARG;
        for (int32_t j = 0; j < n_joints; ++j) {
            const int a = joint_bodies[2 * j], b = joint_bodies[2 * j + 1];
            if (a >= 0 && b >= 0 && scene_of_body[a] != scene_of_body[b]) return OVL_ERR_ARG;
        }
        sc.inv_mass.assign(inv_mass, inv_mass + n);
        sc.jab.assign(joint_bodies, joint_bodies + 2 * (size_t)n_joints);
        std::vector<uint64_t> m(mask, mask + n);
        host_assign_overlap(sc, m);
        std::copy(m.begin(), m.end(), mask);
        return OVL_OK;
    } catch (const std::exception &) {
        return OVL_ERR_ARG;
    }
}
