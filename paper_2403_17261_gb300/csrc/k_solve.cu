// k_solve.cu -- every worker's timestep (Algorithm 1 line 16): projected
// Gauss-Seidel on the MLCP of Eq 1-7 over the worker's active bodies and
// constraints, then integration (Section 3: velocities first, positions with
// the new velocities), writing the worker's copy of each body.
//
// One CTA per worker.  The worker's body velocities live in shared memory
// (32 B per body: (v, 1/m) and (w, 1/I)); workers too large for shared memory
// keep them in a global scratch area instead.  Rows are streamed from HBM/L2
// in colour order: constraints of one colour share no dynamic body, so a
// colour is solved by all threads at once and a barrier separates colours --
// the same result as sweeping the constraints one by one in colour order.
//
// Row model (sphere contact, normal n from a to b, lever arms r_a n and
// -r_b n, tangents t1 and t2 = n x t1):
//   w_n  = n.(v_b - v_a)
//   w_t1 = t1.(v_b - v_a) - t2.(r_a w_a + r_b w_b)
//   w_t2 = t2.(v_b - v_a) + t1.(r_a w_a + r_b w_b)
//   lambda' = clamp(lambda + k (target - w), lo, hi), impulses J^T (lambda' - lambda)
// with lo/hi = [0, inf) for the normal and +-mu lambda_n for the tangents.
// Ball joint: three rows along the world axes, w = (v_b + w_b x r_B - v_a - w_a x r_A)_k.
#include "common.cuh"
#include "kernels.cuh"

namespace ovl {

namespace {

constexpr int NB1 = 2 * OVL_MAX_COLOURS + 1;

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ void axpy(float4 &v, float s, float3 d) { v.x += s * d.x; v.y += s * d.y; v.z += s * d.z; }

struct Body {
    float4 v;  // (v, inverse mass)
    float4 w;  // (omega, inverse inertia)
};

__device__ __forceinline__ Body load_body(const float4 *vel, const float4 *ang, int slot) {
    Body b;
    if (slot >= 0) {
        b.v = vel[slot];
        b.w = ang[slot];
    } else {
        b.v = make_float4(0.f, 0.f, 0.f, 0.f);
        b.w = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return b;
}

__device__ __forceinline__ void store_body(float4 *vel, float4 *ang, int slot, const Body &b) {
    if (slot >= 0) {
        vel[slot] = b.v;
        ang[slot] = b.w;
    }
}

// apply impulse vector lambda (n, t1, t2 components) of a contact
__device__ __forceinline__ void contact_impulse(Body &A, Body &B, float3 n, float3 t1, float3 t2,
                                                float ra, float rb, float ln, float l1, float l2) {
    float3 P = make_float3(n.x * ln + t1.x * l1 + t2.x * l2, n.y * ln + t1.y * l1 + t2.y * l2,
                           n.z * ln + t1.z * l1 + t2.z * l2);
    axpy(A.v, -A.v.w, P);
    axpy(B.v, B.v.w, P);
    // angular: -(r_A x P) on a, (r_B x P) on b with r_A = r_a n, r_B = -r_b n
    float3 L = make_float3(t1.x * l2 - t2.x * l1, t1.y * l2 - t2.y * l1, t1.z * l2 - t2.z * l1);
    axpy(A.w, A.w.w * ra, L);
    axpy(B.w, B.w.w * rb, L);
}

__device__ __forceinline__ void contact_row(Body &A, Body &B, float4 r0, float4 r1, float4 r2,
                                            float4 &lam) {
    const float3 n = f3(r0), t1 = f3(r1);
    const float kn = r0.w, kt = r1.w;
    const float ra = r2.x, rb = r2.y, target = r2.z, mu = r2.w;
    const float3 t2 = cross3(n, t1);
    // normal row
    float3 dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float wn = dot3(n, dv);
    float ln = fmaxf(lam.x + kn * (target - wn), 0.f);
    float d = ln - lam.x;
    lam.x = ln;
    axpy(A.v, -A.v.w * d, n);
    axpy(B.v, B.v.w * d, n);
    const float lim = mu * ln;
    // first tangent
    dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float3 u = make_float3(ra * A.w.x + rb * B.w.x, ra * A.w.y + rb * B.w.y, ra * A.w.z + rb * B.w.z);
    float wt = dot3(t1, dv) - dot3(t2, u);
    float l1 = fminf(fmaxf(lam.y - kt * wt, -lim), lim);
    d = l1 - lam.y;
    lam.y = l1;
    axpy(A.v, -A.v.w * d, t1);
    axpy(B.v, B.v.w * d, t1);
    axpy(A.w, -A.w.w * ra * d, t2);
    axpy(B.w, -B.w.w * rb * d, t2);
    // second tangent
    dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    u = make_float3(ra * A.w.x + rb * B.w.x, ra * A.w.y + rb * B.w.y, ra * A.w.z + rb * B.w.z);
    wt = dot3(t2, dv) + dot3(t1, u);
    float l2 = fminf(fmaxf(lam.z - kt * wt, -lim), lim);
    d = l2 - lam.z;
    lam.z = l2;
    axpy(A.v, -A.v.w * d, t2);
    axpy(B.v, B.v.w * d, t2);
    axpy(A.w, A.w.w * ra * d, t1);
    axpy(B.w, B.w.w * rb * d, t1);
}

__device__ __forceinline__ float joint_w(const Body &A, const Body &B, float3 rA, float3 rB, int ax) {
    float3 ca = cross3(f3(A.w), rA), cb = cross3(f3(B.w), rB);
    float3 rel = make_float3(B.v.x + cb.x - A.v.x - ca.x, B.v.y + cb.y - A.v.y - ca.y,
                             B.v.z + cb.z - A.v.z - ca.z);
    return ax == 0 ? rel.x : (ax == 1 ? rel.y : rel.z);
}

// impulse d along world axis ax at the pivot
__device__ __forceinline__ void joint_impulse(Body &A, Body &B, float3 rA, float3 rB, int ax, float d) {
    float3 e = make_float3(ax == 0 ? d : 0.f, ax == 1 ? d : 0.f, ax == 2 ? d : 0.f);
    axpy(A.v, -A.v.w, e);
    axpy(B.v, B.v.w, e);
    axpy(A.w, -A.w.w, cross3(rA, e));
    axpy(B.w, B.w.w, cross3(rB, e));
}

__device__ __forceinline__ void joint_rows(Body &A, Body &B, float4 r0, float4 r1, float4 r2,
                                           float4 &lam) {
    const float3 rA = f3(r0), rB = f3(r1);
    float k[3] = {r2.x, r2.y, r2.z};
    float t[3] = {r0.w, r1.w, r2.w};
    float l[3] = {lam.x, lam.y, lam.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float w = joint_w(A, B, rA, rB, ax);
        float d = k[ax] * (t[ax] - w);
        l[ax] += d;
        joint_impulse(A, B, rA, rB, ax, d);
    }
    lam = make_float4(l[0], l[1], l[2], lam.w);
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// residual (lambda - clamp(lambda + k (target - w), lo, hi)) / k of a
// contact's three rows, squared and summed; *mx gets the largest magnitude
__device__ __forceinline__ float contact_residual_sq(const Body &A, const Body &B, float4 r0, float4 r1,
                                                     float4 r2, float4 lam, float *mx) {
    const float3 n = f3(r0), t1 = f3(r1);
    const float kn = r0.w, kt = r1.w;
    const float ra = r2.x, rb = r2.y, target = r2.z, mu = r2.w;
    const float3 t2 = cross3(n, t1);
    float3 dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float3 u = make_float3(ra * A.w.x + rb * B.w.x, ra * A.w.y + rb * B.w.y, ra * A.w.z + rb * B.w.z);
    float wn = dot3(n, dv), w1 = dot3(t1, dv) - dot3(t2, u), w2 = dot3(t2, dv) + dot3(t1, u);
    float lim = mu * lam.x;
    float e0 = (lam.x - fmaxf(lam.x + kn * (target - wn), 0.f)) / kn;
    float e1 = (lam.y - clampf(lam.y - kt * w1, -lim, lim)) / kt;
    float e2 = (lam.z - clampf(lam.z - kt * w2, -lim, lim)) / kt;
    *mx = fmaxf(*mx, fmaxf(fabsf(e0), fmaxf(fabsf(e1), fabsf(e2))));
    return e0 * e0 + e1 * e1 + e2 * e2;
}

__device__ __forceinline__ float joint_residual_sq(const Body &A, const Body &B, float4 r0, float4 r1,
                                                   float4 r2, float4 lam, float *mx) {
    const float3 rA = f3(r0), rB = f3(r1);
    float t[3] = {r0.w, r1.w, r2.w};
    float s = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float e = -(t[ax] - joint_w(A, B, rA, rB, ax));   // (lam - (lam + k (t - w))) / k
        *mx = fmaxf(*mx, fabsf(e));
        s += e * e;
    }
    (void)lam;
    return s;
}

__device__ float block_sum(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

template <bool SHARED>
__device__ void solve_worker(const SolveArgs &a, float4 *vel, float4 *ang) {
    __shared__ float red[32];
    __shared__ int stop_flag;
    const int p = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    const int scene = a.part_scene[p];
    const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[scene];
    // velocities after the external force (h f), from the blended state
    for (int s = tid; s < nb; s += T) {
        int b = a.entry_body[a.part_list[b0 + s]];
        float4 v = a.st[4 * b + 2], w = a.st[4 * b + 3];
        vel[s] = make_float4(v.x + h * a.gravity.x, v.y + h * a.gravity.y, v.z + h * a.gravity.z, v.w);
        ang[s] = w;
    }
    __syncthreads();
    const int ncol = a.part_ncol[p];
    const int *off = a.col_off + (size_t)p * NB1;
    // warm start: apply the previous impulses, colour by colour
    for (int c = 0; c < ncol; ++c) {
        const int cb = off[2 * c], jb = off[2 * c + 1], je = off[2 * c + 2];
        for (int r = cb + tid; r < jb; r += T) {
            float4 lam = a.rlam[r];
            if (lam.x == 0.f && lam.y == 0.f && lam.z == 0.f) continue;
            float4 r0 = a.r0[r], r1 = a.r1[r], r2 = a.r2[r];
            int4 r3 = a.r3[r];
            Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
            float3 n = f3(r0), t1 = f3(r1);
            contact_impulse(A, B, n, t1, cross3(n, t1), r2.x, r2.y, lam.x, lam.y, lam.z);
            store_body(vel, ang, r3.x, A);
            store_body(vel, ang, r3.y, B);
        }
        for (int r = jb + tid; r < je; r += T) {
            float4 lam = a.rlam[r];
            float4 r0 = a.r0[r], r1 = a.r1[r];
            int4 r3 = a.r3[r];
            Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
            joint_impulse(A, B, f3(r0), f3(r1), 0, lam.x);
            joint_impulse(A, B, f3(r0), f3(r1), 1, lam.y);
            joint_impulse(A, B, f3(r0), f3(r1), 2, lam.z);
            store_body(vel, ang, r3.x, A);
            store_body(vel, ang, r3.y, B);
        }
        __syncthreads();
    }
    // Gauss-Seidel sweeps
    int it_done = 0;
    if (tid == 0) stop_flag = 0;
    for (int it = 0; it < a.iters; ++it) {
        for (int c = 0; c < ncol; ++c) {
            const int cb = off[2 * c], jb = off[2 * c + 1], je = off[2 * c + 2];
            for (int r = cb + tid; r < jb; r += T) {
                float4 r0 = a.r0[r], r1 = a.r1[r], r2 = a.r2[r];
                int4 r3 = a.r3[r];
                float4 lam = a.rlam[r];
                Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
                contact_row(A, B, r0, r1, r2, lam);
                store_body(vel, ang, r3.x, A);
                store_body(vel, ang, r3.y, B);
                a.rlam[r] = lam;
            }
            for (int r = jb + tid; r < je; r += T) {
                float4 r0 = a.r0[r], r1 = a.r1[r], r2 = a.r2[r];
                int4 r3 = a.r3[r];
                float4 lam = a.rlam[r];
                Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
                joint_rows(A, B, r0, r1, r2, lam);
                store_body(vel, ang, r3.x, A);
                store_body(vel, ang, r3.y, B);
                a.rlam[r] = lam;
            }
            __syncthreads();
        }
        it_done = it + 1;
        if (a.res_tol > 0.f && a.res_check_every > 0 && it_done % a.res_check_every == 0) {
            float sq = 0.f, mx = 0.f;
            const int rb_ = off[0], re_ = off[2 * ncol];
            for (int r = rb_ + tid; r < re_; r += T) {
                float4 r0 = a.r0[r], r1 = a.r1[r], r2 = a.r2[r];
                int4 r3 = a.r3[r];
                float4 lam = a.rlam[r];
                Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
                sq += r3.w == 0 ? contact_residual_sq(A, B, r0, r1, r2, lam, &mx)
                                : joint_residual_sq(A, B, r0, r1, r2, lam, &mx);
            }
            float tot = block_sum(sq, red);
            int nrows = 3 * (re_ - rb_);
            if (tid == 0) stop_flag = (nrows == 0 || sqrtf(tot / nrows) <= a.res_tol) ? 1 : 0;
            __syncthreads();
            if (stop_flag) break;
        }
    }
    // residual of every row at the final iterate
    if (a.flags & OVL_FLAG_RESIDUAL) {
        float sq = 0.f, mx = 0.f;
        const int rb_ = off[0], re_ = off[2 * ncol];
        for (int r = rb_ + tid; r < re_; r += T) {
            float4 r0 = a.r0[r], r1 = a.r1[r], r2 = a.r2[r];
            int4 r3 = a.r3[r];
            float4 lam = a.rlam[r];
            Body A = load_body(vel, ang, r3.x), B = load_body(vel, ang, r3.y);
            sq += r3.w == 0 ? contact_residual_sq(A, B, r0, r1, r2, lam, &mx)
                            : joint_residual_sq(A, B, r0, r1, r2, lam, &mx);
        }
        float tot = block_sum(sq, red);
        if (tid == 0) a.part_res_sq[p] = (double)tot;
    }
    if (tid == 0) a.part_iters[p] = it_done;
    // impulses back in canonical pair order (next step's warm start)
    {
        const int rb_ = off[0], re_ = off[2 * ncol];
        for (int r = rb_ + tid; r < re_; r += T) a.lam_out[a.r3[r].z] = a.rlam[r];
    }
    // integrate: x += h v; q <- normalise(q + h/2 (0, w) (x) q); write this
    // worker's copy of each body
    for (int s = tid; s < nb; s += T) {
        int e = a.part_list[b0 + s];
        int b = a.entry_body[e];
        float4 x = a.st[4 * b], q = a.st[4 * b + 1];
        float4 v = vel[s], w = ang[s];
        float4 xn = make_float4(x.x + h * v.x, x.y + h * v.y, x.z + h * v.z, x.w);
        // (0, w) (x) q = (-w.qv, qw w + w x qv)
        float dqw = -(w.x * q.y + w.y * q.z + w.z * q.w);
        float dqx = q.x * w.x + (w.y * q.w - w.z * q.z);
        float dqy = q.x * w.y + (w.z * q.y - w.x * q.w);
        float dqz = q.x * w.z + (w.x * q.z - w.y * q.y);
        float hh = 0.5f * h;
        float4 qn = make_float4(q.x + hh * dqw, q.y + hh * dqx, q.z + hh * dqy, q.w + hh * dqz);
        float L = sqrtf(qn.x * qn.x + qn.y * qn.y + qn.z * qn.z + qn.w * qn.w);
        qn = make_float4(qn.x / L, qn.y / L, qn.z / L, qn.w / L);
        a.copies[4 * (size_t)e] = xn;
        a.copies[4 * (size_t)e + 1] = qn;
        a.copies[4 * (size_t)e + 2] = v;
        a.copies[4 * (size_t)e + 3] = w;
    }
}

__global__ void k_solve(SolveArgs a) {
    extern __shared__ float4 sm[];
    const int p = blockIdx.x;
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    if (nb <= a.smem_slots) {
        solve_worker<true>(a, sm, sm + nb);
    } else {
        float4 *base = a.scratch + 2 * (size_t)b0;
        solve_worker<false>(a, base, base + nb);
    }
}

}  // namespace

int solve_smem_bytes(int slots) { return slots * 2 * (int)sizeof(float4); }

void launch_solve(const SolveArgs &a, int threads, cudaStream_t s) {
    if (!a.n_parts) return;
    int smem = solve_smem_bytes(a.smem_slots);
    CK(cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_solve<<<a.n_parts, threads, smem, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
