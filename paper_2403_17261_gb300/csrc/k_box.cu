// k_box.cu -- box contact geometry (box-plane, sphere-box, box-box) over
// arrays of pairs, one thread per pair on the GPU, or the same functions on
// the host.  This file is built without FMA contraction on either side, so
// the two runs give the same bits.  The boxes are the bodies of the paper's
// Building and Bridge scenes (Section 6); the step does not use these
// contacts yet.
#include <stdint.h>
#include <string.h>

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

__host__ __device__ void write_points(const PairOut &o, int i, int k, const float3 *p, const float *g, float3 nrm) {
    o.count[i] = k;
    for (int j = 0; j < k; ++j) {
        o.points[12 * (size_t)i + 3 * j] = p[j].x;
        o.points[12 * (size_t)i + 3 * j + 1] = p[j].y;
        o.points[12 * (size_t)i + 3 * j + 2] = p[j].z;
        o.gaps[4 * (size_t)i + j] = g[j];
    }
    o.normal[3 * (size_t)i] = nrm.x;
    o.normal[3 * (size_t)i + 1] = nrm.y;
    o.normal[3 * (size_t)i + 2] = nrm.z;
}

__host__ __device__ void box_plane_one(const BoxPlaneArgs &a, int i) {
    const box::Obb B = obb_of(a.pose + 7 * (size_t)i, a.half + 3 * (size_t)i);
    const float *pl = a.plane + 4 * (size_t)i;
    float3 p[4], n;
    float g[4];
    const int k = box::box_plane(B, make_float4(pl[0], pl[1], pl[2], pl[3]), a.margin, p, g, n);
    write_points(a.o, i, k, p, g, n);
}

__host__ __device__ void sphere_box_one(const SphereBoxArgs &a, int i) {
    const box::Obb B = obb_of(a.pose + 7 * (size_t)i, a.half + 3 * (size_t)i);
    const float *s = a.sphere + 4 * (size_t)i;
    float3 p, n;
    float g;
    const int k = box::sphere_box(make_float3(s[0], s[1], s[2]), s[3], B, a.margin, p, n, g);
    write_points(a.o, i, k, &p, &g, n);
    a.o.gaps[4 * (size_t)i] = g;   // the gap is reported with or without a contact
}

__host__ __device__ void box_box_one(const BoxBoxArgs &a, int i) {
    const box::Obb A = obb_of(a.pose_a + 7 * (size_t)i, a.half_a + 3 * (size_t)i);
    const box::Obb B = obb_of(a.pose_b + 7 * (size_t)i, a.half_b + 3 * (size_t)i);
    float3 p[4], n = make_float3(0.f, 0.f, 0.f);
    float g[4], sep = 0.f;
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
