// k_contacts.cu -- contacts of the blended state (Algorithm 1, contact
// generation, Section 5.4) and the constraint graph G^t (Algorithm 1,
// Section 5.1).
//
// Broadphase: spatial hash grid, one thread per body (cell size >= the
// largest contact distance, so touching spheres sit in neighbouring cells).
// Narrowphase: sphere-sphere (a < b) and sphere-plane.  The contact test and
// the choice of tangent axis decide integers, so they are evaluated in FP32
// with explicit round-to-nearest operations in a fixed order (no fused
// multiply-add):  d2 = (dx*dx + dy*dy) + dz*dz <= (ra + rb + margin)^2 and
// ((nx*px + ny*py) + nz*pz - d) - r <= margin.
//
// Output order is canonical (ascending (a, b), planes numbered after the
// bodies) without a global sort: a per-body count + scan gives each body a
// slot range, and each body sorts its own (few) partners.
//
// Boxes (the paper's Building and Bridge bodies, Section 6): a pair with a
// box end is a candidate when the bounding spheres (radius >= |h|) pass the
// same FP32 test, and the FP64 box geometry of box_geom.cuh (this file is
// built without contraction) then gives 0-4 contacts: the manifold, in
// (a, b, k) order, each with its point.  Counting and writing run the same
// functions on the same inputs, so they agree.
#include <algorithm>

#include "box_geom.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "geom.cuh"

namespace ovl {

namespace {

__device__ __forceinline__ uint32_t cell_hash(int ix, int iy, int iz, int scene, uint32_t mask) {
    uint32_t h = ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^
                 ((uint32_t)iz * 83492791u) ^ ((uint32_t)scene * 2654435761u);
    return h & mask;
}

__global__ void k_cells(const float4 *__restrict__ st, int n, const int *__restrict__ sob,
                        float inv_cs, uint32_t tmask, int4 *__restrict__ cell,
                        int *__restrict__ bucket_count) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        float4 p = st[4 * b];
        int ix = (int)floorf(p.x * inv_cs), iy = (int)floorf(p.y * inv_cs),
            iz = (int)floorf(p.z * inv_cs);
        uint32_t h = cell_hash(ix, iy, iz, sob[b], tmask);
        cell[b] = make_int4(ix, iy, iz, (int)h);
        atomicAdd(&bucket_count[h], 1);
    }
}

__global__ void k_bucket_fill(const int4 *__restrict__ cell, int n, const int *__restrict__ bstart,
                              int *__restrict__ cursor, int *__restrict__ items) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        int h = cell[b].w;
        int slot = atomicAdd(&cursor[h], 1);
        items[bstart[h] + slot] = b;
    }
}

// FP32 sphere-pair test, explicit rounding order
__device__ __forceinline__ bool pair_touches(float4 pa, float4 pb, float margin) {
    float dx = __fsub_rn(pb.x, pa.x), dy = __fsub_rn(pb.y, pa.y), dz = __fsub_rn(pb.z, pa.z);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    float rs = __fadd_rn(__fadd_rn(pa.w, pb.w), margin);
    return d2 <= __fmul_rn(rs, rs);
}

__device__ __forceinline__ float plane_gap(float4 p, float4 pl) {
    float dotp = __fadd_rn(__fadd_rn(__fmul_rn(pl.x, p.x), __fmul_rn(pl.y, p.y)), __fmul_rn(pl.z, p.z));
    return __fsub_rn(__fsub_rn(dotp, pl.w), p.w);
}

// ---- boxes ------------------------------------------------------------------
__device__ __forceinline__ bool is_box(const float4 *half, int b) {
    if (!half) return false;
    const float4 h = half[b];
    return h.x > 0.f || h.y > 0.f || h.z > 0.f;
}

__device__ __forceinline__ box::Obb obb_at(const float4 *st, const float4 *half, int b) {
    const float4 x = st[4 * b], q = st[4 * b + 1], h = half[b];
    return box::make_obb(make_float3(x.x, x.y, x.z), q, make_float3(h.x, h.y, h.z));
}

// contacts of a pair with a box end (a < b, both bodies): points, gaps and
// the normal from a towards b; returns the count (0-4)
__device__ int box_pair(const float4 *st, const float4 *half, const float *radius_w, int a, int b, float margin,
                        double3 *pts, double *gaps, double3 &nrm) {
    const bool ba = is_box(half, a), bb = is_box(half, b);
    if (ba && bb) {
        int axis;
        double sep;
        return box::box_box(obb_at(st, half, a), obb_at(st, half, b), margin, pts, gaps, nrm, axis, sep);
    }
    // one sphere: sphere_box's normal runs from the sphere to the box
    const int sph = ba ? b : a, bx = ba ? a : b;
    const float4 s = st[4 * sph];
    double gap;
    const int hit = box::sphere_box(box::d3(s.x, s.y, s.z), s.w, obb_at(st, half, bx), margin, pts[0], nrm, gap);
    if (sph != a) nrm = box::scl(nrm, -1.0);
    gaps[0] = gap;
    (void)radius_w;
    return hit;
}

// a box against a plane (after the bounding-sphere test)
__device__ int box_plane_pair(const float4 *st, const float4 *half, int a, float4 pl, float margin, double3 *pts,
                              double *gaps, double3 &nrm) {
    return box::box_plane(obb_at(st, half, a), pl, margin, pts, gaps, nrm);
}

__device__ __forceinline__ void write_box_contact(int o, int a, int b, int k, double3 p, double gap, double3 n,
                                                  int2 *c_ab, float4 *c_n, float4 *c_t1, float4 *c_p) {
    const float3 nf = box::to_f(n);
    const float3 t = tangent_from(nf, tangent_axis(nf.x, nf.y, nf.z));
    c_ab[o] = make_int2(a, b);
    c_n[o] = make_float4(nf.x, nf.y, nf.z, (float)gap);
    c_t1[o] = make_float4(t.x, t.y, t.z, 0.f);
    c_p[o] = make_float4((float)p.x, (float)p.y, (float)p.z, __int_as_float(k));
}

// neighbours b > a of body a (sorted ascending) + its plane contacts
// X: the context has boxes.  The box narrow phase (FP64 locals, a large
// stack) is only in the X kernels, so sphere scenes keep a lean kernel.
template <bool X>
__global__ void k_find_pairs(const float4 *__restrict__ st, const float *__restrict__ im, int n,
                             const int *__restrict__ sob, const int *__restrict__ scene_flags,
                             const int4 *__restrict__ cell, const int *__restrict__ bstart,
                             const int *__restrict__ items, uint32_t tmask,
                             const float4 *__restrict__ planes, const int *__restrict__ plane_ptr,
                             const int *__restrict__ plane_list, float margin,
                             int *__restrict__ nb_list, const long long *__restrict__ nb_off,
                             int *__restrict__ nb_count, int *__restrict__ contact_count,
                             int *__restrict__ status, const float4 *__restrict__ half) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const int s = sob[a];
        const float4 pa = st[4 * a];   // .w = radius
        const bool dyn_a = im[a] > 0.0f;
        int cnt = 0;
        int local[OVL_MAX_NEIGH];
        int *const gl = nb_list + nb_off[a];
        const int cap = (int)(nb_off[a + 1] - nb_off[a]);
        bool spilled = false;   // the list continues in gl (more than OVL_MAX_NEIGH neighbours)
        bool overflow = false;
        if (scene_flags[s] & 1) {
            const int4 ca = cell[a];
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        const int cx = ca.x + dx, cy = ca.y + dy, cz = ca.z + dz;
                        const uint32_t h = cell_hash(cx, cy, cz, s, tmask);
                        for (int k = bstart[h]; k < bstart[h + 1]; ++k) {
                            const int b = items[k];
                            if (b <= a) continue;
                            const int4 cb = cell[b];
                            if (cb.x != cx || cb.y != cy || cb.z != cz || sob[b] != s) continue;
                            if (!dyn_a && !(im[b] > 0.0f)) continue;
                            if (!pair_touches(pa, st[4 * b], margin)) continue;
                            if (!spilled && cnt == OVL_MAX_NEIGH && cap > OVL_MAX_NEIGH) {
                                for (int j = 0; j < cnt; ++j) gl[j] = local[j];
                                spilled = true;
                            }
                            if (cnt >= (spilled ? cap : OVL_MAX_NEIGH)) {
                                overflow = true;
                                continue;
                            }
                            // insertion into the sorted list
                            int *lst = spilled ? gl : local;
                            int j = cnt;
                            while (j > 0 && lst[j - 1] > b) {
                                lst[j] = lst[j - 1];
                                --j;
                            }
                            lst[j] = b;
                            ++cnt;
                        }
                    }
        }
        if (overflow) atomicCAS(status, DEV_OK, DEV_ERR_CAPACITY);
        if (!spilled)
            for (int j = 0; j < cnt; ++j) gl[j] = local[j];
        nb_count[a] = cnt;
        // contacts: one per sphere pair, 0-4 per pair with a box end
        int nct = cnt;
        if constexpr (X) {
            const int *lst = spilled ? gl : local;
            nct = 0;
            for (int j = 0; j < cnt; ++j) {
                const int b = lst[j];
                if (!is_box(half, a) && !is_box(half, b)) { ++nct; continue; }
                double3 pts[4], nrm;
                double gaps[4];
                nct += box_pair(st, half, nullptr, a, b, margin, pts, gaps, nrm);
            }
        }
        int np_ = 0;
        if (dyn_a) {
            const bool box_a = X && is_box(half, a);
            for (int k = plane_ptr[s]; k < plane_ptr[s + 1]; ++k) {
                const float4 pl = planes[plane_list[k]];
                if (plane_gap(pa, pl) > margin) continue;   // the (bounding) sphere test
                if (!box_a) { ++np_; continue; }
                if constexpr (X) {
                    double3 pts[4], nrm;
                    double gaps[4];
                    np_ += box_plane_pair(st, half, a, pl, margin, pts, gaps, nrm);
                }
            }
        }
        contact_count[a] = nct + np_;
    }
}

template <bool X>
__global__ void k_write_contacts(const float4 *__restrict__ st, const float *__restrict__ im, int n,
                                 const int *__restrict__ sob, const float4 *__restrict__ planes,
                                 const int *__restrict__ plane_ptr, const int *__restrict__ plane_list,
                                 float margin, const int *__restrict__ nb_list,
                                 const long long *__restrict__ nb_off,
                                 const int *__restrict__ nb_count, const int *__restrict__ cstart,
                                 int2 *__restrict__ c_ab, float4 *__restrict__ c_n,
                                 float4 *__restrict__ c_t1, const float4 *__restrict__ half,
                                 float4 *__restrict__ c_p) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const float4 pa = st[4 * a];
        int o = cstart[a];
        const int cnt = nb_count[a];
        for (int j = 0; j < cnt; ++j) {
            const int b = nb_list[nb_off[a] + j];
            const float4 pb = st[4 * b];
            if constexpr (X) {
                if (is_box(half, a) || is_box(half, b)) {
                    double3 pts[4], nrm;
                    double gaps[4];
                    const int m = box_pair(st, half, nullptr, a, b, margin, pts, gaps, nrm);
                    for (int k = 0; k < m; ++k)
                        write_box_contact(o++, a, b, k, pts[k], gaps[k], nrm, c_ab, c_n, c_t1, c_p);
                    continue;
                }
            }
            float dx = __fsub_rn(pb.x, pa.x), dy = __fsub_rn(pb.y, pa.y), dz = __fsub_rn(pb.z, pa.z);
            float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            float L = __fsqrt_rn(d2);
            float3 nn;
            int k;
            if (L == 0.0f) {
                nn = make_float3(0.f, 0.f, 1.f);
                k = 0;
            } else {
                nn = make_float3(__fdiv_rn(dx, L), __fdiv_rn(dy, L), __fdiv_rn(dz, L));
                k = tangent_axis(nn.x, nn.y, nn.z);
            }
            float3 t = tangent_from(nn, k);
            // The gap from the exact FP64 differences of the FP32 centres and an
            // FP64 square root, rounded once: it enters the speculative target
            // -phi / h, which multiplies an FP32 rounding of |d| (~1e-7 m)
            // into ~1e-5 m/s of velocity.
            const double ex = (double)pb.x - (double)pa.x, ey = (double)pb.y - (double)pa.y,
                         ez = (double)pb.z - (double)pa.z;
            const double L64 = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
            const float phi = (float)((L64 - (double)pa.w) - (double)pb.w);
            c_ab[o] = make_int2(a, b);
            c_n[o] = make_float4(nn.x, nn.y, nn.z, phi);
            c_t1[o] = make_float4(t.x, t.y, t.z, 0.f);
            if (c_p) c_p[o] = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
            ++o;
        }
        if (im[a] > 0.0f) {
            const int s = sob[a];
            const bool box_a = X && is_box(half, a);
            for (int k2 = plane_ptr[s]; k2 < plane_ptr[s + 1]; ++k2) {
                const int pidx = plane_list[k2];
                const float4 pl = planes[pidx];
                if (plane_gap(pa, pl) > margin) continue;   // the FP32 (bounding-sphere) decision
                if constexpr (X) {
                    if (box_a) {
                        double3 pts[4], nrm;
                        double gaps[4];
                        const int m = box_plane_pair(st, half, a, pl, margin, pts, gaps, nrm);
                        for (int k = 0; k < m; ++k)
                            write_box_contact(o++, a, n + pidx, k, pts[k], gaps[k], nrm, c_ab, c_n, c_t1, c_p);
                        continue;
                    }
                }
                // the gap itself from large coordinates: FP64, then rounded once
                const float gap = (float)((double)pl.x * pa.x + (double)pl.y * pa.y +
                                          (double)pl.z * pa.z - (double)pl.w - (double)pa.w);
                // normal from the sphere towards the plane
                float3 nn = make_float3(-pl.x, -pl.y, -pl.z);
                int k = tangent_axis(nn.x, nn.y, nn.z);
                float3 t = tangent_from(nn, k);
                c_ab[o] = make_int2(a, n + pidx);
                c_n[o] = make_float4(nn.x, nn.y, nn.z, gap);
                c_t1[o] = make_float4(t.x, t.y, t.z, 0.f);
                if (c_p) c_p[o] = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
                ++o;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// G^t: undirected edges between two dynamic bodies from contacts and joints
// ---------------------------------------------------------------------------
__global__ void k_edge_degree(const int2 *__restrict__ c_ab, int nc, const int2 *__restrict__ jab,
                              int nj, const float *__restrict__ im, int n, int *__restrict__ deg) {
    int total = nc + nj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int2 e = i < nc ? c_ab[i] : jab[i - nc];
        if (e.x < 0 || e.y < 0 || e.x >= n || e.y >= n || e.x == e.y) continue;
        if (!(im[e.x] > 0.0f) || !(im[e.y] > 0.0f)) continue;
        atomicAdd(&deg[e.x], 1);
        atomicAdd(&deg[e.y], 1);
    }
}

__global__ void k_edge_fill(const int2 *__restrict__ c_ab, int nc, const int2 *__restrict__ jab,
                            int nj, const float *__restrict__ im, int n,
                            const int *__restrict__ tptr, int *__restrict__ cursor,
                            int *__restrict__ tcol) {
    int total = nc + nj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int2 e = i < nc ? c_ab[i] : jab[i - nc];
        if (e.x < 0 || e.y < 0 || e.x >= n || e.y >= n || e.x == e.y) continue;
        if (!(im[e.x] > 0.0f) || !(im[e.y] > 0.0f)) continue;
        tcol[tptr[e.x] + atomicAdd(&cursor[e.x], 1)] = e.y;
        tcol[tptr[e.y] + atomicAdd(&cursor[e.y], 1)] = e.x;
    }
}

// sort each vertex's neighbours and drop duplicates in place
__global__ void k_adj_unique(const int *__restrict__ tptr, int n, int *__restrict__ tcol,
                             int *__restrict__ ucount) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int b = tptr[v], e = tptr[v + 1];
        for (int i = b + 1; i < e; ++i) {
            int x = tcol[i];
            int j = i;
            while (j > b && tcol[j - 1] > x) {
                tcol[j] = tcol[j - 1];
                --j;
            }
            tcol[j] = x;
        }
        int m = 0;
        for (int i = b; i < e; ++i)
            if (i == b || tcol[i] != tcol[i - 1]) tcol[b + m++] = tcol[i];
        ucount[v] = m;
    }
}

__global__ void k_adj_compact(const int *__restrict__ tptr, const int *__restrict__ tcol, int n,
                              const int *__restrict__ row_ptr, int *__restrict__ col) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int m = row_ptr[v + 1] - row_ptr[v];
        for (int k = 0; k < m; ++k) col[row_ptr[v] + k] = tcol[tptr[v] + k];
    }
}

// Load-balance candidates: contacts between two dynamic bodies (all of
// them when the removal branches run), or only those whose worker sets are
// disjoint (activation-only steps: activations only add workers, so a pair
// that shares a worker now can never reach Algorithm 6's activation branch later).
__global__ void k_lb_flags(const int2 *__restrict__ c_ab, int nc, const float *__restrict__ im, int n,
                           const uint64_t *__restrict__ mask, int disjoint_only, int *__restrict__ flag,
                           const float4 *__restrict__ c_p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        int2 e = c_ab[i];
        // a box pair's manifold takes part once (its first point)
        int f = e.y < n && im[e.x] > 0.0f && im[e.y] > 0.0f && !(c_p && __float_as_int(c_p[i].w) != 0);
        if (f && disjoint_only) f = (mask[e.x] & mask[e.y]) == 0ull;
        flag[i] = f;
    }
}

__global__ void k_lb_compact(const int2 *__restrict__ c_ab, int nc, const int *__restrict__ flag,
                             const int *__restrict__ pos, int2 *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = c_ab[i];
}

// ---- gamma-balls for the load balance --------------------------------------
// The vertex set within gamma hops of a root in G^t (the ball an activation of Algorithm 6 adds)
// depends on the graph only, which Algorithm 6 does not change, so it is
// found for every possible root before the sequential pass: one warp per
// body that is an end of a candidate contact, breadth first, level by
// level, with the vertices seen in a shared-memory hash set.  The set is the
// same whatever the discovery order; the pass applies it in any order (each
// vertex's activation and load update are independent).  A ball larger than
// BALL_CAP vertices is left empty (size 0), and the pass searches it itself.
constexpr int BALL_WARPS = 4, BALL_CAP = 512, BALL_HASH = 1024;

// 1 if u was not in the set (and is now), 0 if it was, -1 if the set is full
__device__ __forceinline__ int ball_insert(int *hs, int u) {
    uint32_t h = ((uint32_t)u * 2654435761u) & (BALL_HASH - 1);
    for (int probe = 0; probe < BALL_HASH; ++probe) {
        const int old = atomicCAS(hs + h, -1, u);
        if (old == -1) return 1;
        if (old == u) return 0;
        h = (h + 1) & (BALL_HASH - 1);
    }
    return -1;
}

// the ends of the candidates whose masks are disjoint now (the activation
// branch); those that become disjoint during the pass are rare enough for
// the host to search
// root[v] = 1 marks v once; list[0..*count) the roots (in any order)
__global__ void k_ball_roots(const int2 *__restrict__ ab, int m, const uint64_t *__restrict__ mask,
                             int *__restrict__ root, int *__restrict__ list, int *__restrict__ count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int2 e = ab[i];
        if (mask[e.x] & mask[e.y]) continue;
        if (atomicExch(root + e.x, 1) == 0) list[atomicAdd(count, 1)] = e.x;
        if (atomicExch(root + e.y, 1) == 0) list[atomicAdd(count, 1)] = e.y;
    }
}

// Over the roots list[0..*count): FILL = false: size[v] = |ball(v)| (0 when
// larger than BALL_CAP; size is zero elsewhere); FILL = true: the ball of
// every root v with size[v] > 0 at vtx[start[v]...]
template <bool FILL>
__global__ void __launch_bounds__(BALL_WARPS * 32)
k_balls(const int *__restrict__ list, const int *__restrict__ count, const int *__restrict__ row_ptr,
        const int *__restrict__ col, const int *__restrict__ sob, const int *__restrict__ scene_gamma,
        int *__restrict__ size, const int *__restrict__ start, int *__restrict__ vtx) {
    __shared__ int hs[BALL_WARPS][BALL_HASH];
    __shared__ int lst[BALL_WARPS][BALL_CAP];
    __shared__ int len[BALL_WARPS];
    __shared__ int full[BALL_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *const H = hs[w], *const L = lst[w];
    const int nr = *count;
    for (int j = blockIdx.x * BALL_WARPS + w; j < nr; j += gridDim.x * BALL_WARPS) {
        const int v = list[j];
        if (FILL && size[v] == 0) continue;
        for (int k = lane; k < BALL_HASH; k += 32) H[k] = -1;
        __syncwarp();
        if (lane == 0) {
            ball_insert(H, v);
            L[0] = v;
            len[w] = 1;
            full[w] = 0;
        }
        __syncwarp();
        const int gamma = scene_gamma[sob[v]];
        int lo = 0, hi = 1;
        for (int d = 0; d < gamma && lo < hi; ++d) {
            for (int i = lo; i < hi; ++i) {
                const int x = L[i];
                for (int k = row_ptr[x] + lane; k < row_ptr[x + 1]; k += 32) {
                    const int u = col[k];
                    const int r = ball_insert(H, u);
                    if (r > 0) {
                        const int pos = atomicAdd(&len[w], 1);
                        if (pos < BALL_CAP) L[pos] = u;
                        else full[w] = 1;
                    } else if (r < 0) {
                        full[w] = 1;
                    }
                }
            }
            __syncwarp();
            lo = hi;
            hi = min(len[w], BALL_CAP);
            __syncwarp();
            if (full[w]) break;
        }
        const int total = full[w] ? 0 : len[w];
        if (!FILL) {
            if (lane == 0) size[v] = total;
        } else {
            const int s0 = start[v];
            for (int k = lane; k < total; k += 32) vtx[s0 + k] = L[k];
        }
        __syncwarp();
    }
}

}  // namespace

int grid1d(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

void launch_cells(const ContactArgs &a, cudaStream_t s) {
    k_cells<<<grid1d(a.n, 256), 256, 0, s>>>(a.st, a.n, a.sob, a.inv_cs, a.tmask, a.cell,
                                             a.bucket_count);
    note_launch();
    CK(cudaGetLastError());
}

void launch_bucket_fill(const ContactArgs &a, cudaStream_t s) {
    k_bucket_fill<<<grid1d(a.n, 256), 256, 0, s>>>(a.cell, a.n, a.bucket_start, a.cursor, a.items);
    note_launch();
    CK(cudaGetLastError());
}

void launch_find_pairs(const ContactArgs &a, cudaStream_t s) {
    auto k = a.half ? k_find_pairs<true> : k_find_pairs<false>;
    k<<<grid1d(a.n, 128), 128, 0, s>>>(
        a.st, a.im, a.n, a.sob, a.scene_flags, a.cell, a.bucket_start, a.items, a.tmask, a.planes,
        a.plane_ptr, a.plane_list, a.margin, a.nb_list, a.nb_off, a.nb_count, a.contact_count, a.status, a.half);
    note_launch();
    CK(cudaGetLastError());
}

void launch_write_contacts(const ContactArgs &a, cudaStream_t s) {
    auto k = a.half ? k_write_contacts<true> : k_write_contacts<false>;
    k<<<grid1d(a.n, 128), 128, 0, s>>>(a.st, a.im, a.n, a.sob, a.planes, a.plane_ptr,
                                                      a.plane_list, a.margin, a.nb_list, a.nb_off,
                                                      a.nb_count, a.contact_start, a.c_ab, a.c_n,
                                                      a.c_t1, a.half, a.c_p);
    note_launch();
    CK(cudaGetLastError());
}

void launch_edge_degree(const int2 *c_ab, int nc, const int2 *jab, int nj, const float *im, int n,
                        int *deg, cudaStream_t s) {
    k_edge_degree<<<grid1d(nc + nj, 256), 256, 0, s>>>(c_ab, nc, jab, nj, im, n, deg);
    note_launch();
    CK(cudaGetLastError());
}

void launch_edge_fill(const int2 *c_ab, int nc, const int2 *jab, int nj, const float *im, int n,
                      const int *tptr, int *cursor, int *tcol, cudaStream_t s) {
    k_edge_fill<<<grid1d(nc + nj, 256), 256, 0, s>>>(c_ab, nc, jab, nj, im, n, tptr, cursor, tcol);
    note_launch();
    CK(cudaGetLastError());
}

void launch_adj_unique(const int *tptr, int n, int *tcol, int *ucount, cudaStream_t s) {
    k_adj_unique<<<grid1d(n, 128), 128, 0, s>>>(tptr, n, tcol, ucount);
    note_launch();
    CK(cudaGetLastError());
}

void launch_adj_compact(const int *tptr, const int *tcol, int n, const int *row_ptr, int *col,
                        cudaStream_t s) {
    k_adj_compact<<<grid1d(n, 128), 128, 0, s>>>(tptr, tcol, n, row_ptr, col);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl

namespace ovl {
namespace {

// |P_w| of every worker: one count per set bit of every mask; a block-local
// histogram when the workers fit shared memory
__global__ void k_contact_degree(const int2 *__restrict__ c_ab, int nc, int n, int *__restrict__ deg,
                                 const float4 *__restrict__ c_p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        if (c_p && __float_as_int(c_p[i].w) != 0) continue;   // a box manifold counts once
        const int2 e = c_ab[i];
        atomicAdd(&deg[e.x], 1);
        if (e.y < n) atomicAdd(&deg[e.y], 1);
    }
}

__global__ void k_worker_loads(const uint64_t *mask, const int *sob, const int *part_base,
                               const int *deg, int n, int P, int *loads) {
    extern __shared__ int hist[];
    const bool local = P <= 8192;
    if (local) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) hist[i] = 0;
        __syncthreads();
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        uint64_t m = mask[b];
        if (!m) continue;
        const int base = part_base[sob[b]];
        const int wt = deg ? 1 + deg[b] : 1;
        while (m) {
            const int w = __ffsll((long long)m) - 1;
            m &= m - 1;
            atomicAdd(local ? &hist[base + w] : &loads[base + w], wt);
        }
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < P; i += blockDim.x)
            if (hist[i]) atomicAdd(&loads[i], hist[i]);
    }
}

}  // namespace

void launch_contact_degree(const int2 *c_ab, int nc, int n, int *deg, const float4 *c_p, cudaStream_t s) {
    CK(cudaMemsetAsync(deg, 0, sizeof(int) * (size_t)n, s));
    if (nc <= 0) return;
    k_contact_degree<<<grid1d(nc, 256), 256, 0, s>>>(c_ab, nc, n, deg, c_p);
    note_launch();
    CK(cudaGetLastError());
}

void launch_worker_loads(const uint64_t *mask, const int *sob, const int *part_base, const int *deg, int n,
                         int P, int *loads, cudaStream_t s) {
    CK(cudaMemsetAsync(loads, 0, sizeof(int) * (size_t)P, s));
    if (n <= 0) return;
    const int smem = P <= 8192 ? P * (int)sizeof(int) : 0;
    k_worker_loads<<<std::min(grid1d(n, 256), 152 * 2), 256, smem, s>>>(mask, sob, part_base, deg, n, P, loads);
    note_launch();
    CK(cudaGetLastError());
}

void launch_lb_flags(const int2 *c_ab, int nc, const float *im, int n, const uint64_t *mask,
                     int disjoint_only, int *flag, const float4 *c_p, cudaStream_t s) {
    if (!nc) return;
    k_lb_flags<<<grid1d(nc, 256), 256, 0, s>>>(c_ab, nc, im, n, mask, disjoint_only, flag, c_p);
    note_launch();
    CK(cudaGetLastError());
}
void launch_lb_compact(const int2 *c_ab, int nc, const int *flag, const int *pos, int2 *out,
                       cudaStream_t s) {
    if (!nc) return;
    k_lb_compact<<<grid1d(nc, 256), 256, 0, s>>>(c_ab, nc, flag, pos, out);
    note_launch();
    CK(cudaGetLastError());
}
void launch_ball_roots(const int2 *ab, int m, const uint64_t *mask, int *root, int *list, int *count,
                       cudaStream_t s) {
    if (!m) return;
    k_ball_roots<<<grid1d(m, 256), 256, 0, s>>>(ab, m, mask, root, list, count);
    note_launch();
    CK(cudaGetLastError());
}
void launch_balls(bool fill, int max_roots, const int *list, const int *count, const int *row_ptr, const int *col,
                  const int *sob, const int *scene_gamma, int *size, const int *start, int *vtx, cudaStream_t s) {
    if (max_roots <= 0) return;
    const int blocks = (int)std::min<size_t>(((size_t)max_roots + BALL_WARPS - 1) / BALL_WARPS, 152 * 16);
    if (fill)
        k_balls<true><<<blocks, BALL_WARPS * 32, 0, s>>>(list, count, row_ptr, col, sob, scene_gamma, size, start, vtx);
    else
        k_balls<false><<<blocks, BALL_WARPS * 32, 0, s>>>(list, count, row_ptr, col, sob, scene_gamma, size, start, vtx);
    note_launch();
    CK(cudaGetLastError());
}
}  // namespace ovl
