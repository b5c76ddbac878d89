// geom.cuh -- small geometry shared by the kernels: rotation of a vector by
// a unit quaternion q = (w, x, y, z) stored as float4 (x = w, y..w = vector
// part), and the contact tangent basis.
#pragma once

namespace ovl {

__device__ __forceinline__ float3 quat_rotate(float4 q, float3 v) {
    // v + 2 w (u x v) + 2 u x (u x v), q = (w, u)
    float3 u = make_float3(q.y, q.z, q.w);
    float3 t = make_float3(2.f * (u.y * v.z - u.z * v.y), 2.f * (u.z * v.x - u.x * v.z),
                           2.f * (u.x * v.y - u.y * v.x));
    return make_float3(v.x + q.x * t.x + (u.y * t.z - u.z * t.y),
                       v.y + q.x * t.y + (u.z * t.x - u.x * t.z),
                       v.z + q.x * t.z + (u.x * t.y - u.y * t.x));
}

// tangent axis of a contact: the axis of the smallest |n_k|, scanning x, y,
// z, a later axis winning only when smaller by more than 1e-4 (axis-aligned
// normals tie exactly in two components; the FP64 reference, with the same
// rule, then picks the same axis)
__device__ __forceinline__ int tangent_axis(float nx, float ny, float nz) {
    const float tie = 1e-4f;
    float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
    int k = 0;
    float m = ax;
    if (ay < m - tie) { k = 1; m = ay; }
    if (az < m - tie) { k = 2; }
    return k;
}

// t1 = normalise(e_k - (n . e_k) n), every operation rounded explicitly so
// that kernels built with and without FMA contraction get the same bits
__device__ __forceinline__ float3 tangent_from(float3 n, int k) {
    const float nk = k == 0 ? n.x : (k == 1 ? n.y : n.z);
    float3 t = make_float3(-__fmul_rn(nk, n.x), -__fmul_rn(nk, n.y), -__fmul_rn(nk, n.z));
    if (k == 0) t.x = __fadd_rn(t.x, 1.0f); else if (k == 1) t.y = __fadd_rn(t.y, 1.0f); else t.z = __fadd_rn(t.z, 1.0f);
    const float inv = rsqrtf(__fadd_rn(__fadd_rn(__fmul_rn(t.x, t.x), __fmul_rn(t.y, t.y)), __fmul_rn(t.z, t.z)));
    return make_float3(__fmul_rn(t.x, inv), __fmul_rn(t.y, inv), __fmul_rn(t.z, inv));
}

}  // namespace ovl
