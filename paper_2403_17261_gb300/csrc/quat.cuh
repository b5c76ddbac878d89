// quat.cuh -- rotation of a vector by a unit quaternion q = (w, x, y, z),
// stored as float4 (x = w, y..w = vector part).
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

}  // namespace ovl
