// k_solve.cu -- every worker's timestep (Algorithm 1): projected
// Gauss-Seidel on the MLCP of Eq 1-7 over the worker's active bodies and
// constraints, then integration (Section 3: velocities first, positions with
// the new velocities), writing the worker's copy of each body.
//
// A worker is solved by a group of C CTAs (a thread-block cluster when C > 1).
// Its bodies live in the shared memory of the group (32 B each: v with 1/m,
// w with 1/I; or, when that does not fit, 24 B of v and w with the masses in
// the row records) -- CTA k holds the contiguous slots [k per, (k + 1) per), per =
// ceil(nb / C), and other CTAs reach them through distributed shared memory
// (mapa + ld/st.shared::cluster) -- or, for workers too large for that, in a
// global scratch area solved by one CTA.  Rows are streamed from HBM/L2 in
// colour order: constraints of one colour share no dynamic body, so a colour
// is solved by all CTAs of the group at once and a group barrier separates
// colours -- the same result as sweeping the constraints one by one in colour
// order.  Inside a colour every CTA takes the rows whose first dynamic body
// it holds (the rows are grouped that way beforehand), so most body accesses
// stay in the CTA's own shared memory.  In full-size CTAs (one per SM) with
// the masses in shared memory, a thread loads its next rows' records and
// impulses into registers ahead of use: the next pass's during the current
// one, the next colour's between the two halves of the colour barrier.
//
// Row model (sphere contact, normal n from a to b, lever arms r_a n and
// -r_b n, tangents t1 and t2 = n x t1):
//   w_n  = n.(v_b - v_a)
//   w_t1 = t1.(v_b - v_a) - t2.(r_a w_a + r_b w_b)
//   w_t2 = t2.(v_b - v_a) + t1.(r_a w_a + r_b w_b)
//   lambda' = clamp(lambda + k (target - w), lo, hi), impulses J^T (lambda' - lambda)
// with lo/hi = [0, inf) for the normal and +-mu lambda_n for the tangents.
// Ball joint: three rows along the world axes, w = (v_b + w_b x r_B - v_a - w_a x r_A)_k,
// k = 1 / (1/m_a + 1/m_b + |r_A x e_k|^2 / I_a + |r_B x e_k|^2 / I_b).
//
// Row records (float4 each): contact r0 = (n, slot_b), r1 = (r_a, r_b,
// target, slot_a); joint r0 = (r_A, target_x), r1 = (r_B, target_y), r2 =
// (target_z, 0, slot_a, slot_b); both r3 = (1/m_a, 1/m_b, 1/I_a, 1/I_b),
// read only when the masses are not in shared memory.  Slots are slot codes
// (below).  In a launch with the masses in shared memory a contact has r0 =
// (n, k_t) and r1 = (r_a, r_b, target, slot_a | slot_b << 16) with 16-bit
// codes (such a CTA holds under 8192 slots).  A contact's impulse record is
// (lambda_n, lambda_t1, lambda_t2, k_n).  k_n = 1 / (1/m_a + 1/m_b) and k_t =
// 1 / (1/m_a + 1/m_b + r_a^2 / I_a + r_b^2 / I_b) come from the row build, or
// k_t is formed here from the row's masses with the same operations, so both
// layouts compute the same bits; t1 = normalise(e_k - (n . e_k) n) (k the
// axis of the smallest |n_k|) is formed here.
#include <cooperative_groups.h>

#include "common.cuh"
#include "geom.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace ovl {

namespace {

constexpr int SOLVE_THREADS = 512;

// The file is built without FMA contraction, and its fused multiply-adds are
// written out (fmaf): every instantiation (cluster size, rows per thread,
// slot layout, CTA width) then rounds the same way and gives the same bits.
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x)));
}
__device__ __forceinline__ void axpy(float3 &v, float s, float3 d) {
    v.x = fmaf(s, d.x, v.x);
    v.y = fmaf(s, d.y, v.y);
    v.z = fmaf(s, d.z, v.z);
}
// ra a + rb b
__device__ __forceinline__ float3 lever_sum(float ra, float3 a, float rb, float3 b) {
    return make_float3(fmaf(ra, a.x, rb * b.x), fmaf(ra, a.y, rb * b.y), fmaf(ra, a.z, rb * b.z));
}

struct Body {
    float3 v, w;
    float im, ii;   // inverse mass and inertia (0 for a static end)
};


// ---- body storage --------------------------------------------------------
// A row names its bodies by slot codes: rank << 24 | i, body i of the slot
// range CTA `rank` of the group holds (rank 0 and the worker slot itself
// with one CTA).  A static end (or a body not active in this worker) names
// the zero slot i = per of the row's own CTA: zero velocity, mass and
// inertia, and every impulse leaves it zero, so no row branches on its ends.
// Shared-memory slots per CTA: per + 1.

__device__ __forceinline__ uint32_t code_rank(uint32_t c) { return c >> 24; }
__device__ __forceinline__ uint32_t code_index(uint32_t c) { return c & 0xffffffu; }

// One CTA, shared memory.  kMasses: the slots hold the inverse mass and
// inertia too (else they come with the row).
struct LocalSlots {
    static constexpr bool kMasses = false;
    float4 *A;   // (vx, vy, vz, wx)
    float2 *B;   // (wy, wz)
    __device__ __forceinline__ uint32_t code_of(int s) const { return (uint32_t)s; }
    __device__ __forceinline__ void load(uint32_t c, Body &b) const {
        const uint32_t i = code_index(c);
        const float4 x = A[i];
        const float2 y = B[i];
        b.v = make_float3(x.x, x.y, x.z);
        b.w = make_float3(x.w, y.x, y.y);
    }
    __device__ __forceinline__ void store(uint32_t c, const Body &b) const {
        const uint32_t i = code_index(c);
        A[i] = make_float4(b.v.x, b.v.y, b.v.z, b.w.x);
        B[i] = make_float2(b.w.y, b.w.z);
    }
};

// (v, 1/m) and (w, 1/I) of slot i at S[2i], S[2i + 1]
struct LocalSlotsM {
    static constexpr bool kMasses = true;
    float4 *S;
    __device__ __forceinline__ uint32_t code_of(int s) const { return (uint32_t)s; }
    __device__ __forceinline__ void load(uint32_t c, Body &b) const {
        const uint32_t i = code_index(c);
        const float4 x = S[2 * i], y = S[2 * i + 1];
        b.v = make_float3(x.x, x.y, x.z);
        b.w = make_float3(y.x, y.y, y.z);
        b.im = x.w;
        b.ii = y.w;
    }
    __device__ __forceinline__ void store(uint32_t c, const Body &b) const {
        const uint32_t i = code_index(c);
        S[2 * i] = make_float4(b.v.x, b.v.y, b.v.z, b.im);
        S[2 * i + 1] = make_float4(b.w.x, b.w.y, b.w.z, b.ii);
    }
};

__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// Distributed over the C CTAs of a cluster: the slot range of CTA `rank` is
// in that CTA's shared memory, reached through distributed shared memory
// (mapa + ld/st.shared::cluster).  The accesses are volatile asm, so they
// keep their order among themselves and with the cluster barriers; ordinary
// loads of row records may move around them.
template <int C>
struct ClusterSlots {
    static constexpr bool kMasses = false;
    uint32_t A, B;   // shared-window offsets of this CTA's arrays (same in every CTA)
    uint32_t per;    // slots per CTA
    __device__ __forceinline__ uint32_t code_of(int s) const { return ((uint32_t)s / per) << 24 | (uint32_t)s % per; }
    __device__ __forceinline__ void load(uint32_t c, Body &b) const {
        const uint32_t r = code_rank(c), i = code_index(c);
        const uint32_t a = mapa(A + 16u * i, r), d = mapa(B + 8u * i, r);
        float4 x;
        float2 y;
        asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w) : "r"(a));
        asm volatile("ld.shared::cluster.v2.f32 {%0,%1}, [%2];" : "=f"(y.x), "=f"(y.y) : "r"(d));
        b.v = make_float3(x.x, x.y, x.z);
        b.w = make_float3(x.w, y.x, y.y);
    }
    __device__ __forceinline__ void store(uint32_t c, const Body &b) const {
        const uint32_t r = code_rank(c), i = code_index(c);
        const uint32_t a = mapa(A + 16u * i, r), d = mapa(B + 8u * i, r);
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1,%2,%3,%4};"
                     :: "r"(a), "f"(b.v.x), "f"(b.v.y), "f"(b.v.z), "f"(b.w.x));
        asm volatile("st.shared::cluster.v2.f32 [%0], {%1,%2};" :: "r"(d), "f"(b.w.y), "f"(b.w.z));
    }
};

// the same with the masses: one 32 B slot, one mapa per access
template <int C>
struct ClusterSlotsM {
    static constexpr bool kMasses = true;
    uint32_t S;      // shared-window offset of this CTA's slots (same in every CTA)
    uint32_t per;    // slots per CTA
    __device__ __forceinline__ uint32_t code_of(int s) const { return ((uint32_t)s / per) << 24 | (uint32_t)s % per; }
    __device__ __forceinline__ void load(uint32_t c, Body &b) const {
        const uint32_t a = mapa(S + 32u * code_index(c), code_rank(c));
        float4 x, y;
        asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w) : "r"(a));
        asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(y.x), "=f"(y.y), "=f"(y.z), "=f"(y.w) : "r"(a + 16u));
        b.v = make_float3(x.x, x.y, x.z);
        b.w = make_float3(y.x, y.y, y.z);
        b.im = x.w;
        b.ii = y.w;
    }
    __device__ __forceinline__ void store(uint32_t c, const Body &b) const {
        const uint32_t a = mapa(S + 32u * code_index(c), code_rank(c));
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1,%2,%3,%4};"
                     :: "r"(a), "f"(b.v.x), "f"(b.v.y), "f"(b.v.z), "f"(b.im));
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1,%2,%3,%4};"
                     :: "r"(a + 16u), "f"(b.w.x), "f"(b.w.y), "f"(b.w.z), "f"(b.ii));
    }
};

// A worker too large for shared memory, solved by one CTA in a global
// scratch area of worker slots: a code's slot is rank per + i, and i = per
// is a static end (no zero slot here).
struct GlobalSlots {
    static constexpr bool kMasses = false;
    float4 *A;
    float2 *B;
    uint32_t per;    // slots per CTA of the worker's launch (the codes' ranges)
    __device__ __forceinline__ uint32_t code_of(int s) const { return ((uint32_t)s / per) << 24 | (uint32_t)s % per; }
    __device__ __forceinline__ void load(uint32_t c, Body &b) const {
        const uint32_t i = code_index(c);
        if (i >= per) { b.v = make_float3(0.f, 0.f, 0.f); b.w = b.v; return; }
        const uint32_t s = code_rank(c) * per + i;
        const float4 x = A[s];
        const float2 y = B[s];
        b.v = make_float3(x.x, x.y, x.z);
        b.w = make_float3(x.w, y.x, y.y);
    }
    __device__ __forceinline__ void store(uint32_t c, const Body &b) const {
        const uint32_t i = code_index(c);
        if (i >= per) return;
        const uint32_t s = code_rank(c) * per + i;
        A[s] = make_float4(b.v.x, b.v.y, b.v.z, b.w.x);
        B[s] = make_float2(b.w.y, b.w.z);
    }
};

// One row as the solver reads it: x = r0, y = r1, z = r2 (joints) and m =
// r3 when the slots do not carry the masses.
struct Row {
    float4 x, y, z, m;
    bool joint;
};

template <class S>
__device__ __forceinline__ void fetch_row(const SolveArgs &a, int r, bool joint, Row &w) {
    w.joint = joint;
    w.x = a.r0[r];
    w.y = a.r1[r];
    if (joint) w.z = a.r2[r];
    if (!S::kMasses) w.m = a.r3[r];
}

// a joint's r2 (r0, r1 and r3 come from a RowPre)
__device__ __forceinline__ void fetch_row_rest(const SolveArgs &a, int r, bool joint, Row &w) {
    w.joint = joint;
    if (joint) w.z = a.r2[r];
}

// a 16-bit slot code (rank << 13 | i) as a slot code
__device__ __forceinline__ uint32_t code_from16(uint32_t c) { return (c >> 13) << 24 | (c & 0x1fffu); }

// the slot codes (a, b) of a row: a contact of a launch with the masses in
// shared memory packs both as 16-bit codes in r1.w (its r0.w holds k_t)
template <class S>
__device__ __forceinline__ uint2 row_slots(const Row &w) {
    if (w.joint) return make_uint2(__float_as_uint(w.z.z), __float_as_uint(w.z.w));
    if (S::kMasses) {
        const uint32_t c = __float_as_uint(w.y.w);
        return make_uint2(code_from16(c & 0xffffu), code_from16(c >> 16));
    }
    return make_uint2(__float_as_uint(w.y.w), __float_as_uint(w.x.w));
}

// a static end reads its zero slot (or, without the masses in the slots,
// zero masses from r3)
template <class S>
__device__ __forceinline__ void load_pair(const S &st, const Row &w, Body &A, Body &B) {
    const uint2 slots = row_slots<S>(w);
    st.load(slots.x, A);
    st.load(slots.y, B);
    if (!S::kMasses) { A.im = w.m.x; B.im = w.m.y; A.ii = w.m.z; B.ii = w.m.w; }
}

// k_t of a contact's tangent rows from the bodies' masses and lever radii
__device__ __forceinline__ float contact_kt(const Body &A, const Body &B, float ra, float rb) {
    return __frcp_rn(fmaf(B.ii, rb * rb, fmaf(A.ii, ra * ra, A.im + B.im)));
}

// k_t as the launch has it: in r0.w (masses in shared memory, written by the
// row build with the same operations), or formed from the row's masses
template <class S>
__device__ __forceinline__ float row_kt(const Row &w, const Body &A, const Body &B) {
    return S::kMasses ? w.x.w : contact_kt(A, B, w.y.x, w.y.y);
}

// t1 of a contact, formed from its normal
__device__ __forceinline__ float3 contact_t1(const Row &w) {
    const float3 n = make_float3(w.x.x, w.x.y, w.x.z);
    return tangent_from(n, tangent_axis(n.x, n.y, n.z));
}

template <class S>
__device__ __forceinline__ void store_pair(const S &st, uint2 slots, const Body &A, const Body &B) {
    st.store(slots.x, A);
    st.store(slots.y, B);
}

// ---- rows ----------------------------------------------------------------
// impulses (n, t1, t2) components (ln, l1, l2) of a contact
__device__ __forceinline__ void contact_impulse(Body &A, Body &B, float3 n, float3 t1, float3 t2,
                                                float ra, float rb, float ln, float l1, float l2) {
    float3 P = make_float3(fmaf(n.x, ln, fmaf(t1.x, l1, t2.x * l2)), fmaf(n.y, ln, fmaf(t1.y, l1, t2.y * l2)),
                           fmaf(n.z, ln, fmaf(t1.z, l1, t2.z * l2)));
    axpy(A.v, -A.im, P);
    axpy(B.v, B.im, P);
    // angular: -(r_A x P) on a, (r_B x P) on b with r_A = r_a n, r_B = -r_b n
    float3 L = make_float3(fmaf(t1.x, l2, -(t2.x * l1)), fmaf(t1.y, l2, -(t2.y * l1)), fmaf(t1.z, l2, -(t2.z * l1)));
    axpy(A.w, A.ii * ra, L);
    axpy(B.w, B.ii * rb, L);
}

__device__ __forceinline__ void contact_row(Body &A, Body &B, float4 r0, float4 r1, float3 t1, float kn,
                                            float kt, float mu, float4 &lam) {
    const float3 n = f3(r0);
    const float ra = r1.x, rb = r1.y, target = r1.z;
    const float3 t2 = cross3(n, t1);
    // normal row
    float3 dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float ln = fmaxf(fmaf(kn, target - dot3(n, dv), lam.x), 0.f);
    float d = ln - lam.x;
    lam.x = ln;
    axpy(A.v, -A.im * d, n);
    axpy(B.v, B.im * d, n);
    const float lim = mu * ln;
    // first tangent
    dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float3 u = lever_sum(ra, A.w, rb, B.w);
    float wt = dot3(t1, dv) - dot3(t2, u);
    float l1 = fminf(fmaxf(fmaf(-kt, wt, lam.y), -lim), lim);
    d = l1 - lam.y;
    lam.y = l1;
    axpy(A.v, -A.im * d, t1);
    axpy(B.v, B.im * d, t1);
    axpy(A.w, -A.ii * ra * d, t2);
    axpy(B.w, -B.ii * rb * d, t2);
    // second tangent
    dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    u = lever_sum(ra, A.w, rb, B.w);
    wt = dot3(t2, dv) + dot3(t1, u);
    float l2 = fminf(fmaxf(fmaf(-kt, wt, lam.z), -lim), lim);
    d = l2 - lam.z;
    lam.z = l2;
    axpy(A.v, -A.im * d, t2);
    axpy(B.v, B.im * d, t2);
    axpy(A.w, A.ii * ra * d, t1);
    axpy(B.w, B.ii * rb * d, t1);
}

__device__ __forceinline__ float joint_w(const Body &A, const Body &B, float3 rA, float3 rB, int ax) {
    float3 ca = cross3(A.w, rA), cb = cross3(B.w, rB);
    float3 rel = make_float3(B.v.x + cb.x - A.v.x - ca.x, B.v.y + cb.y - A.v.y - ca.y,
                             B.v.z + cb.z - A.v.z - ca.z);
    return ax == 0 ? rel.x : (ax == 1 ? rel.y : rel.z);
}

// impulse d along world axis ax at the pivot
__device__ __forceinline__ void joint_impulse(Body &A, Body &B, float3 rA, float3 rB, int ax, float d) {
    float3 e = make_float3(ax == 0 ? d : 0.f, ax == 1 ? d : 0.f, ax == 2 ? d : 0.f);
    axpy(A.v, -A.im, e);
    axpy(B.v, B.im, e);
    axpy(A.w, -A.ii, cross3(rA, e));
    axpy(B.w, B.ii, cross3(rB, e));
}

// k_kk = 1 / (1/m_a + 1/m_b + |r_A x e_k|^2 / I_a + |r_B x e_k|^2 / I_b)
__device__ __forceinline__ float joint_k(const Body &A, const Body &B, float3 rA, float3 rB, int ax) {
    float a2 = ax == 0 ? fmaf(rA.y, rA.y, rA.z * rA.z) : (ax == 1 ? fmaf(rA.x, rA.x, rA.z * rA.z) : fmaf(rA.x, rA.x, rA.y * rA.y));
    float b2 = ax == 0 ? fmaf(rB.y, rB.y, rB.z * rB.z) : (ax == 1 ? fmaf(rB.x, rB.x, rB.z * rB.z) : fmaf(rB.x, rB.x, rB.y * rB.y));
    return __frcp_rn(fmaf(B.ii, b2, fmaf(A.ii, a2, A.im + B.im)));
}

__device__ __forceinline__ void joint_rows(Body &A, Body &B, float4 r0, float4 r1, float4 r2, float4 &lam) {
    const float3 rA = f3(r0), rB = f3(r1);
    float t[3] = {r0.w, r1.w, r2.x};
    float l[3] = {lam.x, lam.y, lam.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float d = joint_k(A, B, rA, rB, ax) * (t[ax] - joint_w(A, B, rA, rB, ax));
        l[ax] += d;
        joint_impulse(A, B, rA, rB, ax, d);
    }
    lam = make_float4(l[0], l[1], l[2], lam.w);
}

// one constraint's rows in the sweep
template <class S>
__device__ __forceinline__ void solve_row(Body &A, Body &B, const Row &w, float mu, float4 &lam) {
    if (w.joint) {
        joint_rows(A, B, w.x, w.y, w.z, lam);
    } else {
        contact_row(A, B, w.x, w.y, contact_t1(w), lam.w, row_kt<S>(w, A, B), mu, lam);
    }
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// ---- full rows (a box end: general lever arms and inertia responses) -------
// Only the kernels of contexts with boxes (X) hold this code: in the sphere
// kernels its registers would add to the rows' loop, which then spills.
template <bool X>
__device__ __forceinline__ bool is_full(const SolveArgs &a, int r) { return X && a.row_full[r]; }

// impulse dl along direction i of a full row
__device__ __forceinline__ void full_impulse(const float4 *F, int i, float imA, float imB, Body &A, Body &B,
                                             float dl) {
    const float3 d = f3(F[i]);
    axpy(A.v, -imA * dl, d);
    axpy(B.v, imB * dl, d);
    axpy(A.w, -dl, f3(F[6 + i]));
    axpy(B.w, dl, f3(F[12 + i]));
}

__device__ __forceinline__ float full_w(const float4 *F, int i, const Body &A, const Body &B) {
    const float3 dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    return dot3(f3(F[i]), dv) + (dot3(f3(F[9 + i]), B.w) - dot3(f3(F[3 + i]), A.w));
}

// the three rows of a constraint with a box end: contact (normal >= 0,
// tangents within +-mu lambda_n) or ball joint (unbounded)
__device__ void full_rows(const SolveArgs &a, int r, bool joint, Body &A, Body &B, float mu, float4 &lam) {
    const float4 *F = a.rfull + (size_t)r * FULL_ROW_WORDS;
    const float imA = F[15].x, imB = F[15].y;
    float l[3] = {lam.x, lam.y, lam.z};
    for (int i = 0; i < 3; ++i) {
        const float k = F[3 + i].w, target = F[i].w;
        float ln = fmaf(k, target - full_w(F, i, A, B), l[i]);
        if (!joint) ln = i == 0 ? fmaxf(ln, 0.f) : fminf(fmaxf(ln, -mu * l[0]), mu * l[0]);
        const float dl = ln - l[i];
        l[i] = ln;
        full_impulse(F, i, imA, imB, A, B, dl);
    }
    lam = make_float4(l[0], l[1], l[2], lam.w);
}

__device__ void full_warm(const SolveArgs &a, int r, Body &A, Body &B, float4 lam) {
    const float4 *F = a.rfull + (size_t)r * FULL_ROW_WORDS;
    const float imA = F[15].x, imB = F[15].y;
    full_impulse(F, 0, imA, imB, A, B, lam.x);
    full_impulse(F, 1, imA, imB, A, B, lam.y);
    full_impulse(F, 2, imA, imB, A, B, lam.z);
}

// a row of the sweep: full (box end) or plain
template <class S, bool X>
__device__ __forceinline__ void solve_any(const SolveArgs &a, int r, Body &A, Body &B, const Row &w, float mu,
                                          float4 &lam) {
    if (is_full<X>(a, r)) full_rows(a, r, w.joint, A, B, mu, lam);
    else solve_row<S>(A, B, w, mu, lam);
}

__device__ float full_residual_sq(const SolveArgs &a, int r, bool joint, const Body &A, const Body &B, float mu,
                                  float4 lam) {
    const float4 *F = a.rfull + (size_t)r * FULL_ROW_WORDS;
    const float l[3] = {lam.x, lam.y, lam.z};
    float s = 0.f;
    for (int i = 0; i < 3; ++i) {
        const float k = F[3 + i].w;
        float p = l[i] + k * (F[i].w - full_w(F, i, A, B));
        if (!joint) p = i == 0 ? fmaxf(p, 0.f) : clampf(p, -mu * l[0], mu * l[0]);
        const float e = k > 0.f ? (l[i] - p) / k : 0.f;
        s += e * e;
    }
    return s;
}

// residual (lambda - clamp(lambda + k (target - w), lo, hi)) / k of a row
// group, squared and summed
__device__ __forceinline__ float contact_residual_sq(const Body &A, const Body &B, float4 r0, float4 r1,
                                                     float3 t1, float kn, float kt, float mu, float4 lam) {
    const float3 n = f3(r0);
    const float ra = r1.x, rb = r1.y, target = r1.z;
    const float3 t2 = cross3(n, t1);
    float3 dv = make_float3(B.v.x - A.v.x, B.v.y - A.v.y, B.v.z - A.v.z);
    float3 u = lever_sum(ra, A.w, rb, B.w);
    float wn = dot3(n, dv), w1 = dot3(t1, dv) - dot3(t2, u), w2 = dot3(t2, dv) + dot3(t1, u);
    float lim = mu * lam.x;
    float e0 = (lam.x - fmaxf(lam.x + kn * (target - wn), 0.f)) / kn;
    float e1 = (lam.y - clampf(lam.y - kt * w1, -lim, lim)) / kt;
    float e2 = (lam.z - clampf(lam.z - kt * w2, -lim, lim)) / kt;
    return e0 * e0 + e1 * e1 + e2 * e2;
}

__device__ __forceinline__ float joint_residual_sq(const Body &A, const Body &B, float4 r0, float4 r1,
                                                   float4 r2) {
    const float3 rA = f3(r0), rB = f3(r1);
    float t[3] = {r0.w, r1.w, r2.x};
    float s = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float e = joint_w(A, B, rA, rB, ax) - t[ax];   // (lam - (lam + k (t - w))) / k
        s += e * e;
    }
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

template <int C>
__device__ __forceinline__ void group_sync() {
    if (C == 1) __syncthreads();
    else cg::this_cluster().sync();
}

// The group barrier in two halves: arrive releases this thread's body
// stores, wait acquires the other threads'.  Loads issued between the two
// wait for neither.
template <int C>
__device__ __forceinline__ void group_arrive() {
    if (C > 1) asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
template <int C>
__device__ __forceinline__ void group_wait() {
    if (C == 1) __syncthreads();
    else asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// r0, r1 (and r3 without the masses in shared memory) and the impulse of a
// thread's next two rows of a bucket (rows r and r + T of a bucket ending at
// ce).  Row records are read-only during the solve and a row's impulse is
// read and written by one thread only, so they may be loaded a pass, or a
// colour, ahead.
struct RowPre {
    float4 x0, y0, m0, l0, x1, y1, m1, l1;
};

template <class S>
__device__ __forceinline__ void pre_rows(const SolveArgs &a, int r, int ce, int T, RowPre &p) {
    // every field is written on every path, so the previous values are dead
    // once used
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    p.x0 = p.y0 = p.m0 = p.l0 = p.x1 = p.y1 = p.m1 = p.l1 = z;
    if (r < ce) {
        p.x0 = a.r0[r];
        p.y0 = a.r1[r];
        if (!S::kMasses) p.m0 = a.r3[r];
        p.l0 = a.rlam[r];
    }
    if (r + T < ce) {
        p.x1 = a.r0[r + T];
        p.y1 = a.r1[r + T];
        if (!S::kMasses) p.m1 = a.r3[r + T];
        p.l1 = a.rlam[r + T];
    }
}

// group-wide sum of one value per thread (every thread gets the total)
template <int C>
__device__ float group_sum(float v, float *red, float *slot) {
    float t = block_sum(v, red);
    if (C == 1) return t;
    if (threadIdx.x == 0) *slot = t;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    float tot = 0.f;
    for (int r = 0; r < C; ++r) tot += *cl.map_shared_rank(slot, r);
    cl.sync();
    return tot;
}

// row buckets of colour c: off[(c OWNER_RANKS + k) 2 + kind], contacts then
// joints, for the owner ranks k in [k0, k1)
// Row buckets of this CTA: bucket k of colour c spans rows [tab[c cs + 2k],
// tab[c cs + 2k + 2]), contacts up to tab[c cs + 2k + 1], for k < nbk.
struct Buckets {
    const int *tab;
    int cs, nbk;
};

template <class S, bool X>
__device__ float rows_residual_sq(const SolveArgs &a, const S &st, const Buckets &bk, int ncol, float mu,
                                  int tid, int T) {
    float sq = 0.f;
    for (int c = 0; c < ncol; ++c)
        for (int k = 0; k < bk.nbk; ++k) {
            const int o = c * bk.cs + 2 * k;
            const int jb = bk.tab[o + 1], ce = bk.tab[o + 2];
            for (int r = bk.tab[o] + tid; r < ce; r += T) {
                Row w;
                fetch_row<S>(a, r, r >= jb, w);
                const float4 lam = a.rlam[r];
                Body A, B;
                load_pair(st, w, A, B);
                if (is_full<X>(a, r)) {
                    sq += full_residual_sq(a, r, w.joint, A, B, mu, lam);
                } else if (w.joint) {
                    sq += joint_residual_sq(A, B, w.x, w.y, w.z);
                } else {
                    sq += contact_residual_sq(A, B, w.x, w.y, contact_t1(w), lam.w, row_kt<S>(w, A, B), mu, lam);
                }
            }
        }
    return sq;
}

// One worker solved by a group of C CTAs.  CTA `rank` holds the body slots
// [rank per, min(nb, (rank + 1) per)) and, in every colour, takes the rows of
// its owner bucket, thread tid the rows tid, tid + T, ..., U of them at a
// time.  With C = 1 (one CTA, or the global-memory path) the CTA holds every
// slot and takes every bucket.
template <int C, int U, bool P, bool X, class S>
__device__ void solve_worker(const SolveArgs &a, const S &st, int p, int rank, int per, const Buckets &bk,
                             int row0, int row1) {
    __shared__ float red[32];
    __shared__ float part_sum;
    const int tid = threadIdx.x, T = blockDim.x;
    const int g = rank * T + tid, G = C * T;
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    const int s_lo = C == 1 ? 0 : rank * per, s_hi = C == 1 ? nb : min(nb, (rank + 1) * per);
    const int scene = a.part_scene[p];
    const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[scene];
    const float mu = a.scene_mu[scene];
    // velocities after the external force (h f), from the blended state; each
    // CTA loads the slots it holds
    for (int s = s_lo + tid; s < s_hi; s += T) {
        int b = a.entry_body[a.part_list[b0 + s]];
        float4 v = a.st[4 * b + 2], w = a.st[4 * b + 3];
        Body x;
        x.v = make_float3(v.x + h * a.gravity.x, v.y + h * a.gravity.y, v.z + h * a.gravity.z);
        x.w = make_float3(w.x, w.y, w.z);
        x.im = v.w;
        x.ii = w.w;
        st.store(st.code_of(s), x);
    }
    // this CTA's zero slot (static ends of its rows)
    if (tid == 0) {
        Body z;
        z.v = make_float3(0.f, 0.f, 0.f);
        z.w = z.v;
        z.im = 0.f;
        z.ii = 0.f;
        st.store((uint32_t)rank << 24 | (uint32_t)per, z);
    }
    group_sync<C>();
    const int ncol = a.part_ncol[p];
    // warm start: apply the previous impulses, colour by colour
    for (int c = 0; c < ncol; ++c) {
      for (int k = 0; k < bk.nbk; ++k) {
        const int o = c * bk.cs + 2 * k;
        const int jb = bk.tab[o + 1], ce = bk.tab[o + 2];
        for (int r = bk.tab[o] + tid; r < ce; r += T) {
            float4 lam = a.rlam[r];
            if (lam.x == 0.f && lam.y == 0.f && lam.z == 0.f) continue;
            Row w;
            fetch_row<S>(a, r, r >= jb, w);
            Body A, B;
            load_pair(st, w, A, B);
            if (is_full<X>(a, r)) {
                full_warm(a, r, A, B, lam);
            } else if (!w.joint) {
                const float3 t1 = contact_t1(w);
                const float3 n = f3(w.x);
                contact_impulse(A, B, n, t1, cross3(n, t1), w.y.x, w.y.y, lam.x, lam.y, lam.z);
            } else {
                joint_impulse(A, B, f3(w.x), f3(w.y), 0, lam.x);
                joint_impulse(A, B, f3(w.x), f3(w.y), 1, lam.y);
                joint_impulse(A, B, f3(w.x), f3(w.y), 2, lam.z);
            }
            store_pair(st, row_slots<S>(w), A, B);
        }
      }
      group_sync<C>();
    }
    // Gauss-Seidel sweeps.  P (full-size CTAs, one per SM, two rows per
    // thread): a pass takes r0, r1 (r3) and the impulses of its rows from
    // registers loaded ahead, at the end of the previous pass or, for a
    // colour's first pass, between the two halves of the previous colour's
    // barrier.  (Measured: 4 % faster there, 7 % slower in the 256-thread CTAs
    // that share an SM, which keep the plain loop.)
    int it_done = 0;
    constexpr bool piped = P && U == 2;
    const bool ahead = piped && bk.nbk == 1;
    RowPre pf;
    if (ahead && a.iters > 0 && ncol > 0) pre_rows<S>(a, bk.tab[0] + tid, bk.tab[2], T, pf);
    for (int it = 0; it < a.iters; ++it) {
        for (int c = 0; c < ncol; ++c) {
          for (int k = 0; k < bk.nbk; ++k) {
            const int o = c * bk.cs + 2 * k;
            const int jb = bk.tab[o + 1], ce = bk.tab[o + 2];
            int r = bk.tab[o] + tid;
            if constexpr (piped) {
                RowPre cur;
                if (ahead) cur = pf;
                else pre_rows<S>(a, r, ce, T, cur);
                // two rows of the colour at once (independent: no shared body)
                for (; r + T < ce; r += 2 * T) {
                    const int q = r + T;
                    Row u, w;
                    u.x = cur.x0; u.y = cur.y0; u.m = cur.m0;
                    w.x = cur.x1; w.y = cur.y1; w.m = cur.m1;
                    fetch_row_rest(a, r, r >= jb, u);
                    fetch_row_rest(a, q, q >= jb, w);
                    float4 xl = cur.l0, yl = cur.l1;
                    Body A, B, D, E;
                    load_pair(st, u, A, B);
                    load_pair(st, w, D, E);
                    solve_any<S, X>(a, r, A, B, u, mu, xl);
                    solve_any<S, X>(a, q, D, E, w, mu, yl);
                    store_pair(st, row_slots<S>(u), A, B);
                    store_pair(st, row_slots<S>(w), D, E);
                    a.rlam[r] = xl;
                    a.rlam[q] = yl;
                    pre_rows<S>(a, r + 2 * T, ce, T, cur);
                }
                if (r < ce) {
                    Row w;
                    w.x = cur.x0; w.y = cur.y0; w.m = cur.m0;
                    fetch_row_rest(a, r, r >= jb, w);
                    float4 lam = cur.l0;
                    Body A, B;
                    load_pair(st, w, A, B);
                    solve_any<S, X>(a, r, A, B, w, mu, lam);
                    store_pair(st, row_slots<S>(w), A, B);
                    a.rlam[r] = lam;
                }
            } else {
                if (U == 2) {
                    // two rows of the colour at once (independent: no shared body)
                    for (; r + T < ce; r += 2 * T) {
                        const int q = r + T;
                        Row u, w;
                        fetch_row<S>(a, r, r >= jb, u);
                        fetch_row<S>(a, q, q >= jb, w);
                        float4 xl = a.rlam[r], yl = a.rlam[q];
                        Body A, B, D, E;
                        load_pair(st, u, A, B);
                        load_pair(st, w, D, E);
                        solve_any<S, X>(a, r, A, B, u, mu, xl);
                        solve_any<S, X>(a, q, D, E, w, mu, yl);
                        store_pair(st, row_slots<S>(u), A, B);
                        store_pair(st, row_slots<S>(w), D, E);
                        a.rlam[r] = xl;
                        a.rlam[q] = yl;
                    }
                }
                for (; r < ce; r += T) {
                    Row w;
                    fetch_row<S>(a, r, r >= jb, w);
                    float4 lam = a.rlam[r];
                    Body A, B;
                    load_pair(st, w, A, B);
                    solve_any<S, X>(a, r, A, B, w, mu, lam);
                    store_pair(st, row_slots<S>(w), A, B);
                    a.rlam[r] = lam;
                }
            }
          }
          if (ahead) {
              group_arrive<C>();
              const bool last = c + 1 == ncol;
              if (!last || it + 1 < a.iters) {
                  const int on = last ? 0 : (c + 1) * bk.cs;
                  pre_rows<S>(a, bk.tab[on] + tid, bk.tab[on + 2], T, pf);
              }
              group_wait<C>();
          } else {
              group_sync<C>();
          }
        }
        it_done = it + 1;
        if (a.res_tol > 0.f && a.res_check_every > 0 && it_done % a.res_check_every == 0 && it_done < a.iters) {
            float tot = group_sum<C>(rows_residual_sq<S, X>(a, st, bk, ncol, mu, tid, T), red, &part_sum);
            int nrows = 3 * (row1 - row0);
            if (nrows == 0 || sqrtf(tot / nrows) <= a.res_tol) break;   // the same total in every CTA
        }
    }
    // residual of every row at the final iterate
    if (a.flags & OVL_FLAG_RESIDUAL) {
        float tot = group_sum<C>(rows_residual_sq<S, X>(a, st, bk, ncol, mu, tid, T), red, &part_sum);
        if (rank == 0 && tid == 0) a.part_res_sq[p] = (double)tot;
    }
    if (rank == 0 && tid == 0) a.part_iters[p] = it_done;
    // impulses back in canonical pair order (next step's warm start)
    for (int r = row0 + g; r < row1; r += G) a.lam_out[a.rpair[r]] = a.rlam[r];
    // integrate: x += h v; q <- normalise(q + h/2 (0, w) (x) q); write this
    // worker's copy of each body the CTA holds
    for (int s = s_lo + tid; s < s_hi; s += T) {
        int e = a.part_list[b0 + s];
        int b = a.entry_body[e];
        float4 x = a.st[4 * b], q = a.st[4 * b + 1], v0 = a.st[4 * b + 2], w0 = a.st[4 * b + 3];
        Body y;
        st.load(st.code_of(s), y);
        float3 v = y.v, w = y.w;
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
        a.copies[4 * (size_t)e + 2] = make_float4(v.x, v.y, v.z, v0.w);
        a.copies[4 * (size_t)e + 3] = make_float4(w.x, w.y, w.z, w0.w);
    }
    // no CTA may leave while another can still reach its shared memory
    if (C > 1) group_sync<C>();
}

// C CTAs per worker; a worker's slots are spread over their shared memory when
// they fit (ceil(nb / C) <= smem_slots), else CTA rank 0 solves it alone with
// its body state in the global scratch area.  M: the shared-memory slots hold
// the masses (32 B per slot; else 24 B, and rows carry the masses in r3).
// P: rows loaded ahead (launches of SOLVE_THREADS threads, one CTA per SM).
template <int C, int U, bool M, bool P, bool X>
__global__ void __launch_bounds__(SOLVE_THREADS, U == 1 ? 2 : 1) k_solve(SolveArgs a) {
    extern __shared__ float4 sm[];
    const int rank = C == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int p = a.order ? (int)a.order[blockIdx.x / C] : (int)(blockIdx.x / C);
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    const int per = (nb + C - 1) / C;
    // this CTA's row buckets (three offsets per colour), read in every colour
    // of every sweep
    const int *goff = a.col_off + (size_t)p * OWNER_NB;
    __shared__ int boff[3 * OVL_MAX_COLOURS];
    const int ncol = a.part_ncol[p];
    for (int i = threadIdx.x; i < 3 * ncol; i += blockDim.x)
        boff[i] = goff[((i / 3) * OWNER_RANKS + rank) * 2 + i % 3];
    __syncthreads();
    const int row0 = goff[0], row1 = goff[OWNER_NB - 1];
    if (per <= a.smem_slots) {
        // per + 1 slots: the CTA's range and its zero slot
        float4 *A = sm;
        if (M) {
            if (C == 1) {
                LocalSlotsM st{A};
                solve_worker<C, U, P, X>(a, st, p, rank, per, Buckets{boff, 3, 1}, row0, row1);
            } else {
                ClusterSlotsM<C> st{(uint32_t)__cvta_generic_to_shared(A), (uint32_t)per};
                solve_worker<C, U, P, X>(a, st, p, rank, per, Buckets{boff, 3, 1}, row0, row1);
            }
        } else {
            float2 *B = reinterpret_cast<float2 *>(sm + per + 1);
            if (C == 1) {
                LocalSlots st{A, B};
                solve_worker<C, U, P, X>(a, st, p, rank, per, Buckets{boff, 3, 1}, row0, row1);
            } else {
                ClusterSlots<C> st{(uint32_t)__cvta_generic_to_shared(A), (uint32_t)__cvta_generic_to_shared(B),
                                   (uint32_t)per};
                solve_worker<C, U, P, X>(a, st, p, rank, per, Buckets{boff, 3, 1}, row0, row1);
            }
        }
    } else if (rank == 0) {
        // one CTA takes the whole worker: every owner bucket of every colour
        GlobalSlots st{a.scratch + (size_t)b0, reinterpret_cast<float2 *>(a.scratch + (size_t)a.n_entries) + b0,
                       (uint32_t)per};
        solve_worker<1, U, false, X>(a, st, p, 0, nb, Buckets{goff, 2 * OWNER_RANKS, OWNER_RANKS}, row0, row1);
    }
}

}  // namespace

int solve_slot_bytes(bool masses) { return (int)(masses ? 2 * sizeof(float4) : sizeof(float4) + sizeof(float2)); }

// a CTA's slots and its zero slot
int solve_smem_bytes(int slots, bool masses) { return (slots + 1) * solve_slot_bytes(masses); }

template <int C, int U, bool M, bool P, bool X>
static void launch_solve_c(const SolveArgs &a, int threads, cudaStream_t s) {
    int smem = solve_smem_bytes(a.smem_slots, M);
    CK(cudaFuncSetAttribute(k_solve<C, U, M, P, X>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_parts * C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_solve<C, U, M, P, X>, a));
    note_launch();
}

template <int U, bool M, bool P, bool X = false>
static void launch_solve_u(const SolveArgs &a, int threads, int cluster, cudaStream_t s) {
    switch (cluster) {
        case 8: launch_solve_c<8, U, M, P, X>(a, threads, s); break;
        case 6: launch_solve_c<6, U, M, P, X>(a, threads, s); break;
        case 4: launch_solve_c<4, U, M, P, X>(a, threads, s); break;
        case 3: launch_solve_c<3, U, M, P, X>(a, threads, s); break;
        case 2: launch_solve_c<2, U, M, P, X>(a, threads, s); break;
        default: launch_solve_c<1, U, M, P, X>(a, threads, s); break;
    }
}

void launch_solve(const SolveArgs &a, int threads, int cluster, int unroll, bool masses, cudaStream_t s) {
    if (!a.n_parts) return;
    if (threads > SOLVE_THREADS) threads = SOLVE_THREADS;
    if (a.row_full) {
        // a context with boxes: the kernels that hold the full rows (two rows
        // per thread, no rows loaded ahead; one CTA per SM at 512 threads)
        if (masses) launch_solve_u<2, true, false, true>(a, threads, cluster, s);
        else launch_solve_u<2, false, false, true>(a, threads, cluster, s);
    } else if (unroll == 2) {
        // a full-size CTA (one per SM) loads rows ahead
        if (threads == SOLVE_THREADS) {
            if (masses) launch_solve_u<2, true, true>(a, threads, cluster, s);
            else launch_solve_u<2, false, true>(a, threads, cluster, s);
        } else if (masses) {
            launch_solve_u<2, true, false>(a, threads, cluster, s);
        } else {
            launch_solve_u<2, false, false>(a, threads, cluster, s);
        }
    } else {
        if (masses) launch_solve_u<1, true, false>(a, threads, cluster, s);
        else launch_solve_u<1, false, false>(a, threads, cluster, s);
    }
    CK(cudaGetLastError());
}

// shared-memory bytes a CTA can use when `per_sm` CTAs share an SM, for the
// unroll variant's register budget
int solve_ctas_per_sm(int unroll) { return unroll == 2 ? 1 : 2; }

}  // namespace ovl
