// k_box.cu -- box contact geometry (box-plane, sphere-box, box-box) over
// arrays of pairs, one thread per pair on the GPU, or the same functions on
// the host, computed in FP64 from the FP32 inputs and rounded once.  This
// file is built without FMA contraction on either side, so the two runs
// give the same bits.  The boxes are the bodies of the paper's
// Building and Bridge scenes (Section 6); the step does not use these
// contacts yet.
#include <stdint.h>
#include <string.h>

#include <cmath>

#include <vector>

#include "box_geom.cuh"
#include "common.cuh"
#include "ovl.h"

namespace ovl {
namespace {

// pose: x, y, z, then the quaternion w, x, y, z
__host__ __device__ __forceinline__ box::Obb obb_of(const float *pose, const float *half) {
    return box::make_obb(make_float3(pose[0], pose[1], pose[2]), make_float4(pose[3], pose[4], pose[5], pose[6]),
                         make_float3(half[0], half[1], half[2]));
}

struct PairOut {
    int32_t *count;
    float *points, *gaps, *normal;   // [n][4][3], [n][4], [n][3]
    int32_t *axis;                   // box-box only
};

struct BoxPlaneArgs {
    int n;
    const float *pose, *half, *plane;
    float margin;
    PairOut o;
};
struct SphereBoxArgs {
    int n;
    const float *sphere, *pose, *half;
    float margin;
    PairOut o;
};
struct BoxBoxArgs {
    int n;
    const float *pose_a, *half_a, *pose_b, *half_b;
    float margin;
    PairOut o;
};

// the FP64 results, each rounded once to FP32
__host__ __device__ void write_points(const PairOut &o, int i, int k, const double3 *p, const double *g, double3 nrm) {
    o.count[i] = k;
    for (int j = 0; j < k; ++j) {
        o.points[12 * (size_t)i + 3 * j] = (float)p[j].x;
        o.points[12 * (size_t)i + 3 * j + 1] = (float)p[j].y;
        o.points[12 * (size_t)i + 3 * j + 2] = (float)p[j].z;
        o.gaps[4 * (size_t)i + j] = (float)g[j];
    }
    o.normal[3 * (size_t)i] = (float)nrm.x;
    o.normal[3 * (size_t)i + 1] = (float)nrm.y;
    o.normal[3 * (size_t)i + 2] = (float)nrm.z;
}

__host__ __device__ void box_plane_one(const BoxPlaneArgs &a, int i) {
    const box::Obb B = obb_of(a.pose + 7 * (size_t)i, a.half + 3 * (size_t)i);
    const float *pl = a.plane + 4 * (size_t)i;
    double3 p[4], n;
    double g[4];
    const int k = box::box_plane(B, make_float4(pl[0], pl[1], pl[2], pl[3]), a.margin, p, g, n);
    write_points(a.o, i, k, p, g, n);
}

__host__ __device__ void sphere_box_one(const SphereBoxArgs &a, int i) {
    const box::Obb B = obb_of(a.pose + 7 * (size_t)i, a.half + 3 * (size_t)i);
    const float *s = a.sphere + 4 * (size_t)i;
    double3 p, n;
    double g;
    const int k = box::sphere_box(box::d3(s[0], s[1], s[2]), s[3], B, a.margin, p, n, g);
    write_points(a.o, i, k, &p, &g, n);
    a.o.gaps[4 * (size_t)i] = (float)g;   // the gap is reported with or without a contact
}

__host__ __device__ void box_box_one(const BoxBoxArgs &a, int i) {
    const box::Obb A = obb_of(a.pose_a + 7 * (size_t)i, a.half_a + 3 * (size_t)i);
    const box::Obb B = obb_of(a.pose_b + 7 * (size_t)i, a.half_b + 3 * (size_t)i);
    double3 p[4], n = box::d3(0.0, 0.0, 0.0);
    double g[4], sep = 0.0;
    int axis = -1;
    const int k = box::box_box(A, B, a.margin, p, g, n, axis, sep);
    write_points(a.o, i, k, p, g, n);
    a.o.axis[i] = axis;
}

struct BoxStepArgs {
    int n;
    const float *pose, *half, *inv_mass, *plane;
    float mu, dt, gx, gy, gz, erp, slop, margin;
    int iters;
    float *vel;      // [n][6] v, omega (in/out)
    int32_t *count;  // [n]
    float *lam;      // [n][12]
};

__host__ __device__ void box_step_one(const BoxStepArgs &a, int i) {
    const box::Obb B = obb_of(a.pose + 7 * (size_t)i, a.half + 3 * (size_t)i);
    const float *pl = a.plane + 4 * (size_t)i;
    float *vw = a.vel + 6 * (size_t)i;
    float3 v = make_float3(vw[0], vw[1], vw[2]), w = make_float3(vw[3], vw[4], vw[5]);
    float lam[12] = {0.f};
    const int k = box::box_plane_step(B, a.inv_mass[i], make_float4(pl[0], pl[1], pl[2], pl[3]), a.mu, a.dt,
                                      make_float3(a.gx, a.gy, a.gz), a.erp, a.slop, a.margin, a.iters, v, w, lam);
    vw[0] = v.x; vw[1] = v.y; vw[2] = v.z;
    vw[3] = w.x; vw[4] = w.y; vw[5] = w.z;
    a.count[i] = k;
    for (int j = 0; j < 12; ++j) a.lam[12 * (size_t)i + j] = j < 3 * k ? lam[j] : 0.f;
}

// ---- all contacts of a scene with boxes --------------------------------------
struct SceneArgs {
    int n, n_planes;
    const float *state, *radius, *inv_mass, *half, *planes;   // [n][13], [n], [n], [n][3], [np][4]
    const int32_t *sob, *scene_flags, *plane_scene;
    float margin;
    // outputs (write pass): from offset[a], in (a, b, k) order
    const int64_t *offset;
    int32_t *count_of;                  // count pass: contacts of each body a
    int32_t *ab, *k;
    float *phi, *normal, *point;
};

__host__ __device__ __forceinline__ bool is_box3(const float *h) { return h[0] > 0.f || h[1] > 0.f || h[2] > 0.f; }

__host__ __device__ __forceinline__ float3 pos_of(const float *st) { return make_float3(st[0], st[1], st[2]); }

// contacts of body a with the bodies after it in its scene, then with its
// scene's planes; write == false only counts
__host__ __device__ int scene_contacts_of(const SceneArgs &A, int a, bool write) {
    const float *sa = A.state + 13 * (size_t)a;
    const float3 ca = pos_of(sa);
    const int s = A.sob[a];
    const bool boxa = is_box3(A.half + 3 * (size_t)a);
    int64_t o = write ? A.offset[a] : 0;
    int cnt = 0;
    auto put = [&](int b, int kk, double gap, double3 n, double3 p) {
        if (write) {
            A.ab[2 * o] = a; A.ab[2 * o + 1] = b; A.k[o] = kk; A.phi[o] = (float)gap;
            A.normal[3 * o] = (float)n.x; A.normal[3 * o + 1] = (float)n.y; A.normal[3 * o + 2] = (float)n.z;
            A.point[3 * o] = (float)p.x; A.point[3 * o + 1] = (float)p.y; A.point[3 * o + 2] = (float)p.z;
            ++o;
        }
        ++cnt;
    };
    if (A.scene_flags[s] & 1) {
        for (int b = a + 1; b < A.n; ++b) {
            if (A.sob[b] != s || (A.inv_mass[a] == 0.f && A.inv_mass[b] == 0.f)) continue;
            const float *sb = A.state + 13 * (size_t)b;
            const float3 cb = pos_of(sb);
            if (!box::spheres_touch(ca, cb, A.radius[a], A.radius[b], A.margin)) continue;
            const bool boxb = is_box3(A.half + 3 * (size_t)b);
            if (!boxa && !boxb) {
                // two spheres: one contact, the gap in FP64
                const double3 d = box::sub(box::to_d(cb), box::to_d(ca));
                const double L = sqrt(box::dot(d, d));
                const double3 n = L > 0.0 ? box::scl(d, 1.0 / L) : box::d3(0.0, 0.0, 1.0);
                put(b, 0, (L - (double)A.radius[a]) - (double)A.radius[b], n,
                    box::add(box::to_d(ca), box::scl(n, (double)A.radius[a])));
                continue;
            }
            double3 pts[4], n;
            double gaps[4];
            if (boxa && boxb) {
                const box::Obb Ba = obb_of(sa, A.half + 3 * (size_t)a), Bb = obb_of(sb, A.half + 3 * (size_t)b);
                int axis;
                double sep;
                const int m = box::box_box(Ba, Bb, A.margin, pts, gaps, n, axis, sep);
                for (int i = 0; i < m; ++i) put(b, i, gaps[i], n, pts[i]);
            } else {
                // sphere_box's normal runs from the sphere to the box
                const int sph = boxa ? b : a, bx = boxa ? a : b;
                const float *ss = A.state + 13 * (size_t)sph, *sx = A.state + 13 * (size_t)bx;
                const box::Obb B = obb_of(sx, A.half + 3 * (size_t)bx);
                double gap;
                if (box::sphere_box(box::to_d(pos_of(ss)), A.radius[sph], B, A.margin, pts[0], n, gap))
                    put(b, 0, gap, sph == a ? n : box::scl(n, -1.0), pts[0]);
            }
        }
    }
    if (A.inv_mass[a] > 0.f)
        for (int p = 0; p < A.n_planes; ++p) {
            if (A.plane_scene[p] != s) continue;
            const float4 pl = make_float4(A.planes[4 * p], A.planes[4 * p + 1], A.planes[4 * p + 2], A.planes[4 * p + 3]);
            if (!box::sphere_plane_touch(ca, A.radius[a], pl, A.margin)) continue;
            if (boxa) {
                double3 pts[4], n;
                double gaps[4];
                const int m = box::box_plane(obb_of(sa, A.half + 3 * (size_t)a), pl, A.margin, pts, gaps, n);
                for (int i = 0; i < m; ++i) put(A.n + p, i, gaps[i], n, pts[i]);
            } else {
                const double dotp = ((double)pl.x * ca.x + (double)pl.y * ca.y) + (double)pl.z * ca.z;
                const double3 n = box::d3(-pl.x, -pl.y, -pl.z);
                put(A.n + p, 0, (dotp - (double)pl.w) - (double)A.radius[a], n,
                    box::add(box::to_d(ca), box::scl(n, (double)A.radius[a])));
            }
        }
    if (!write) A.count_of[a] = cnt;
    return cnt;
}

__global__ void k_scene_contacts(SceneArgs A, int write) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < A.n) scene_contacts_of(A, a, write != 0);
}

__global__ void k_box_plane_step(BoxStepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) box_step_one(a, i);
}

__global__ void k_box_plane(BoxPlaneArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) box_plane_one(a, i);
}
__global__ void k_sphere_box(SphereBoxArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) sphere_box_one(a, i);
}
__global__ void k_box_box(BoxBoxArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) box_box_one(a, i);
}

// device copies of host arrays for one call; freed on every exit path
struct DevArena {
    std::vector<void *> held;
    ~DevArena() {
        for (void *p : held) cudaFree(p);
    }
    template <class T>
    T *in(const T *h, size_t count) {
        T *d = nullptr;
        CK(cudaMalloc(&d, sizeof(T) * (count ? count : 1)));
        held.push_back(d);
        if (count) CK(cudaMemcpy(d, h, sizeof(T) * count, cudaMemcpyHostToDevice));
        return d;
    }
    template <class T>
    T *out(size_t count) {
        T *d = nullptr;
        CK(cudaMalloc(&d, sizeof(T) * (count ? count : 1)));
        held.push_back(d);
        CK(cudaMemset(d, 0, sizeof(T) * (count ? count : 1)));
        return d;
    }
};

template <class T>
void fetch(T *h, const T *d, size_t count) {
    if (count) CK(cudaMemcpy(h, d, sizeof(T) * count, cudaMemcpyDeviceToHost));
}

void clear_out(int n, int32_t *count, float *points, float *gaps, float *normal, int32_t *axis) {
    memset(count, 0, sizeof(int32_t) * (size_t)n);
    memset(points, 0, sizeof(float) * 12 * (size_t)n);
    memset(gaps, 0, sizeof(float) * 4 * (size_t)n);
    memset(normal, 0, sizeof(float) * 3 * (size_t)n);
    if (axis) memset(axis, 0, sizeof(int32_t) * (size_t)n);
}

template <class F>
ovl_status guard(F &&f) {
    try {
        return f();
    } catch (const CudaError &) {
        return OVL_ERR_CUDA;
    } catch (...) {
        return OVL_ERR_ARG;
    }
}

}  // namespace
}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_box_plane_contacts(int32_t n, const float *pose, const float *half, const float *plane,
                                             float margin, int32_t on_gpu, int32_t *count, float *points,
                                             float *gaps, float *normal) {
    if (n < 0 || (n > 0 && (!pose || !half || !plane || !count || !points || !gaps || !normal))) return OVL_ERR_ARG;
    return guard([&]() -> ovl_status {
        clear_out(n, count, points, gaps, normal, nullptr);
        if (n == 0) return OVL_OK;
        BoxPlaneArgs a{n, pose, half, plane, margin, {count, points, gaps, normal, nullptr}};
        if (!on_gpu) {
            for (int i = 0; i < n; ++i) box_plane_one(a, i);
            return OVL_OK;
        }
        DevArena d;
        BoxPlaneArgs g{n, d.in(pose, 7 * (size_t)n), d.in(half, 3 * (size_t)n), d.in(plane, 4 * (size_t)n), margin,
                       {d.out<int32_t>(n), d.out<float>(12 * (size_t)n), d.out<float>(4 * (size_t)n),
                        d.out<float>(3 * (size_t)n), nullptr}};
        k_box_plane<<<(n + 127) / 128, 128>>>(g);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        fetch(count, g.o.count, n);
        fetch(points, g.o.points, 12 * (size_t)n);
        fetch(gaps, g.o.gaps, 4 * (size_t)n);
        fetch(normal, g.o.normal, 3 * (size_t)n);
        return OVL_OK;
    });
}

extern "C" ovl_status ovl_sphere_box_contacts(int32_t n, const float *sphere, const float *pose, const float *half,
                                              float margin, int32_t on_gpu, int32_t *count, float *points,
                                              float *gaps, float *normal) {
    if (n < 0 || (n > 0 && (!sphere || !pose || !half || !count || !points || !gaps || !normal))) return OVL_ERR_ARG;
    return guard([&]() -> ovl_status {
        clear_out(n, count, points, gaps, normal, nullptr);
        if (n == 0) return OVL_OK;
        SphereBoxArgs a{n, sphere, pose, half, margin, {count, points, gaps, normal, nullptr}};
        if (!on_gpu) {
            for (int i = 0; i < n; ++i) sphere_box_one(a, i);
            return OVL_OK;
        }
        DevArena d;
        SphereBoxArgs g{n, d.in(sphere, 4 * (size_t)n), d.in(pose, 7 * (size_t)n), d.in(half, 3 * (size_t)n), margin,
                        {d.out<int32_t>(n), d.out<float>(12 * (size_t)n), d.out<float>(4 * (size_t)n),
                         d.out<float>(3 * (size_t)n), nullptr}};
        k_sphere_box<<<(n + 127) / 128, 128>>>(g);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        fetch(count, g.o.count, n);
        fetch(points, g.o.points, 12 * (size_t)n);
        fetch(gaps, g.o.gaps, 4 * (size_t)n);
        fetch(normal, g.o.normal, 3 * (size_t)n);
        return OVL_OK;
    });
}

extern "C" ovl_status ovl_box_box_contacts(int32_t n, const float *pose_a, const float *half_a, const float *pose_b,
                                           const float *half_b, float margin, int32_t on_gpu, int32_t *count,
                                           float *points, float *gaps, float *normal, int32_t *axis) {
    if (n < 0 || (n > 0 && (!pose_a || !half_a || !pose_b || !half_b || !count || !points || !gaps || !normal ||
                            !axis)))
        return OVL_ERR_ARG;
    return guard([&]() -> ovl_status {
        clear_out(n, count, points, gaps, normal, axis);
        if (n == 0) return OVL_OK;
        BoxBoxArgs a{n, pose_a, half_a, pose_b, half_b, margin, {count, points, gaps, normal, axis}};
        if (!on_gpu) {
            for (int i = 0; i < n; ++i) box_box_one(a, i);
            return OVL_OK;
        }
        DevArena d;
        BoxBoxArgs g{n, d.in(pose_a, 7 * (size_t)n), d.in(half_a, 3 * (size_t)n), d.in(pose_b, 7 * (size_t)n),
                     d.in(half_b, 3 * (size_t)n), margin,
                     {d.out<int32_t>(n), d.out<float>(12 * (size_t)n), d.out<float>(4 * (size_t)n),
                      d.out<float>(3 * (size_t)n), d.out<int32_t>(n)}};
        k_box_box<<<(n + 127) / 128, 128>>>(g);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        fetch(count, g.o.count, n);
        fetch(points, g.o.points, 12 * (size_t)n);
        fetch(gaps, g.o.gaps, 4 * (size_t)n);
        fetch(normal, g.o.normal, 3 * (size_t)n);
        fetch(axis, g.o.axis, n);
        return OVL_OK;
    });
}

extern "C" ovl_status ovl_box_plane_step(int32_t n, const float *pose, const float *half, const float *inv_mass,
                                         const float *plane, float mu, float dt, const float *gravity, float erp,
                                         float slop, float margin, int32_t iters, int32_t on_gpu, float *vel,
                                         int32_t *count, float *lam) {
    if (n < 0 || iters < 0 || !gravity ||
        (n > 0 && (!pose || !half || !inv_mass || !plane || !vel || !count || !lam)))
        return OVL_ERR_ARG;
    return guard([&]() -> ovl_status {
        if (n == 0) return OVL_OK;
        BoxStepArgs a{n, pose, half, inv_mass, plane, mu, dt, gravity[0], gravity[1], gravity[2], erp, slop, margin,
                      iters, vel, count, lam};
        if (!on_gpu) {
            for (int i = 0; i < n; ++i) box_step_one(a, i);
            return OVL_OK;
        }
        DevArena d;
        BoxStepArgs g = a;
        g.pose = d.in(pose, 7 * (size_t)n);
        g.half = d.in(half, 3 * (size_t)n);
        g.inv_mass = d.in(inv_mass, (size_t)n);
        g.plane = d.in(plane, 4 * (size_t)n);
        g.vel = d.in(vel, 6 * (size_t)n);
        g.count = d.out<int32_t>(n);
        g.lam = d.out<float>(12 * (size_t)n);
        k_box_plane_step<<<(n + 127) / 128, 128>>>(g);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        fetch(vel, g.vel, 6 * (size_t)n);
        fetch(count, g.count, n);
        fetch(lam, g.lam, 12 * (size_t)n);
        return OVL_OK;
    });
}

extern "C" ovl_status ovl_box_scene_contacts(int32_t n, const float *state13, const float *radius,
                                             const float *inv_mass, const float *half, const int32_t *scene_of_body,
                                             int32_t n_scenes, const int32_t *scene_flags, int32_t n_planes,
                                             const float *planes, const int32_t *plane_scene, float margin,
                                             int32_t on_gpu, int64_t cap, int64_t *total, int32_t *ab, int32_t *k,
                                             float *phi, float *normal, float *point) {
    if (n < 0 || n_planes < 0 || n_scenes < 1 || cap < 0 || !total || !scene_flags ||
        (n > 0 && (!state13 || !radius || !inv_mass || !half || !scene_of_body)) ||
        (n_planes > 0 && (!planes || !plane_scene)) || (cap > 0 && (!ab || !k || !phi || !normal || !point)))
        return OVL_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (scene_of_body[i] < 0 || scene_of_body[i] >= n_scenes) return OVL_ERR_ARG;
    // a NaN or negative extent would otherwise read as a sphere
    for (size_t i = 0; i < 3 * (size_t)n; ++i)
        if (!(half[i] >= 0.f) || !std::isfinite(half[i])) return OVL_ERR_ARG;
    return guard([&]() -> ovl_status {
        *total = 0;
        if (n == 0) return OVL_OK;
        std::vector<int32_t> cnt(n);
        std::vector<int64_t> off(n + 1, 0);
        SceneArgs A{n, n_planes, state13, radius, inv_mass, half, planes, scene_of_body, scene_flags, plane_scene,
                    margin, nullptr, cnt.data(), nullptr, nullptr, nullptr, nullptr, nullptr};
        if (!on_gpu) {
            for (int a = 0; a < n; ++a) scene_contacts_of(A, a, false);
            for (int a = 0; a < n; ++a) off[a + 1] = off[a] + cnt[a];
            *total = off[n];
            if (off[n] > cap) return OVL_ERR_CAPACITY;
            A.offset = off.data(); A.ab = ab; A.k = k; A.phi = phi; A.normal = normal; A.point = point;
            for (int a = 0; a < n; ++a) scene_contacts_of(A, a, true);
            return OVL_OK;
        }
        DevArena d;
        SceneArgs G = A;
        G.state = d.in(state13, 13 * (size_t)n);
        G.radius = d.in(radius, (size_t)n);
        G.inv_mass = d.in(inv_mass, (size_t)n);
        G.half = d.in(half, 3 * (size_t)n);
        G.sob = d.in(scene_of_body, (size_t)n);
        G.scene_flags = d.in(scene_flags, (size_t)n_scenes);
        G.planes = d.in(planes, 4 * (size_t)n_planes);
        G.plane_scene = d.in(plane_scene, (size_t)n_planes);
        G.count_of = d.out<int32_t>(n);
        k_scene_contacts<<<(n + 127) / 128, 128>>>(G, 0);
        CK(cudaGetLastError());
        fetch(cnt.data(), G.count_of, n);
        for (int a = 0; a < n; ++a) off[a + 1] = off[a] + cnt[a];
        *total = off[n];
        if (off[n] > cap) return OVL_ERR_CAPACITY;
        if (off[n] == 0) return OVL_OK;
        const size_t m = (size_t)off[n];
        G.offset = d.in(off.data(), (size_t)n + 1);
        G.ab = d.out<int32_t>(2 * m);
        G.k = d.out<int32_t>(m);
        G.phi = d.out<float>(m);
        G.normal = d.out<float>(3 * m);
        G.point = d.out<float>(3 * m);
        k_scene_contacts<<<(n + 127) / 128, 128>>>(G, 1);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        fetch(ab, G.ab, 2 * m);
        fetch(k, G.k, m);
        fetch(phi, G.phi, m);
        fetch(normal, G.normal, 3 * m);
        fetch(point, G.point, 3 * m);
        return OVL_OK;
    });
}
