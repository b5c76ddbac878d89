// k_blend.cu -- the weights and the blend of Algorithm 1.
//
// D(o,i) (Eq 16): distance in G^t from an overlap body o to the nearest body
// active only in worker i, searched up to beta (Algorithm 5).  Instead of one
// search per overlap body, one level-synchronous BFS runs from all sources
// at once: a queue item is (body, worker), level 0 holds every body with
// W_b = {i} as (b, i), and a (body, worker) bit marks the pairs already
// reached.  The level at which (o, i) is first reached is exactly
// min over sources of G(o, b); the order in which threads reach it does not
// matter.
//
// Blend (Algorithm 4, Eq 11-15): weights proportional to 1/D (workers not met
// within beta weigh 0; a body that met none gets uniform weights), copies
// summed in ascending worker order, a copy's quaternion negated when its
// dot product with the lowest worker's copy is negative, then normalised.
// Every worker integrated its copy from the same blended state, x_i = x + h v_i
// (Algorithm 1), so Eq 11 equals x + h sum w_i v_i; the
// position is formed that way, which rounds once in FP32 instead of twice.
// Bodies in one worker take their copy unchanged.
#include "common.cuh"
#include "kernels.cuh"
#include "geom.cuh"

namespace ovl {

namespace {

__device__ __forceinline__ long long vbit(const GeoArgs &a, int b, int w) {
    int s = a.sob[b];
    int bs = a.body_base[s + 1] - a.body_base[s];
    return a.vb_base[s] + (long long)w * bs + (b - a.body_base[s]);
}

__device__ __forceinline__ bool claim(uint32_t *visited, long long bit) {
    uint32_t m = 1u << (bit & 31);
    uint32_t old = atomicOr(&visited[bit >> 5], m);
    return !(old & m);
}

__device__ __forceinline__ void enqueue(int *tail, uint32_t *queue, uint32_t item) {
    // warp-aggregated append
    unsigned active = __activemask();
    int leader = __ffs(active) - 1;
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(tail, __popc(active));
    base = __shfl_sync(active, base, leader);
    queue[base + __popc(active & ((1u << lane) - 1u))] = item;
}

__global__ void k_geo_sources(GeoArgs a) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.n; b += gridDim.x * blockDim.x) {
        uint64_t m = a.mask[b];
        if (__popcll(m) != 1) continue;
        int w = __ffsll((long long)m) - 1;
        claim(a.visited, vbit(a, b, w));
        enqueue(&a.qctl[0], a.queue, ((uint32_t)b << 6) | (uint32_t)w);
    }
}

// qctl[1 + L] = first queue index of level L
__global__ void k_geo_mark(int *qctl, int level) { qctl[1 + level] = qctl[0]; }

__global__ void k_geo_level(GeoArgs a, int level) {
    const int start = a.qctl[1 + level - 1], end = a.qctl[1 + level];
    // one warp per frontier item, lanes over its neighbours
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int it = start + gw; it < end; it += warps) {
        uint32_t item = a.queue[it];
        int u = (int)(item >> 6), w = (int)(item & 63u);
        int beta = a.scene_beta[a.sob[u]];
        if (level > beta) continue;
        for (int k = a.row_ptr[u] + lane; k < a.row_ptr[u + 1]; k += 32) {
            int v = a.col[k];
            if (!claim(a.visited, vbit(a, v, w))) continue;
            uint64_t mv = a.mask[v];
            if (__popcll(mv) >= 2 && (mv >> w & 1ull)) {
                int e = a.entry_ptr[v] + __popcll(mv & ((1ull << w) - 1ull));
                a.D[e] = (uint8_t)level;
            }
            if (level < beta) enqueue(&a.qctl[0], a.queue, ((uint32_t)v << 6) | (uint32_t)w);
        }
    }
}

__global__ void k_blend(BlendArgs a) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.n; b += gridDim.x * blockDim.x) {
        const int e0 = a.entry_ptr[b], k = a.entry_ptr[b + 1] - e0;
        float4 o0, o1, o2, o3;
        if (k == 0) {                       // static body: unchanged
            o0 = a.st_in[4 * b]; o1 = a.st_in[4 * b + 1]; o2 = a.st_in[4 * b + 2]; o3 = a.st_in[4 * b + 3];
        } else if (k == 1) {                // one worker: its copy as is
            o0 = a.copies[4 * (size_t)e0]; o1 = a.copies[4 * (size_t)e0 + 1];
            o2 = a.copies[4 * (size_t)e0 + 2]; o3 = a.copies[4 * (size_t)e0 + 3];
            a.weight[e0] = 1.0f;
        } else {
            // Eq 15 weights from inverse geodesic distances
            float s = 0.f;
            for (int i = 0; i < k; ++i) {
                uint8_t d = a.D[e0 + i];
                s += d != 255 ? 1.0f / (float)d : 0.f;
            }
            const float4 x0 = a.copies[4 * (size_t)e0], q0 = a.copies[4 * (size_t)e0 + 1];
            const float4 xs = a.st_in[4 * b];
            const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[a.sob[b]];
            float3 v = make_float3(0.f, 0.f, 0.f), w = v;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = 0; i < k; ++i) {
                const size_t e = (size_t)(e0 + i);
                uint8_t d = a.D[e];
                float wi = (s > 0.f && !a.uniform) ? (d != 255 ? (1.0f / (float)d) / s : 0.f)
                                                   : 1.0f / (float)k;
                a.weight[e] = wi;
                float4 qi = a.copies[4 * e + 1], vi = a.copies[4 * e + 2], wv = a.copies[4 * e + 3];
                v.x += wi * vi.x; v.y += wi * vi.y; v.z += wi * vi.z;
                w.x += wi * wv.x; w.y += wi * wv.y; w.z += wi * wv.z;
                float dq = qi.x * q0.x + qi.y * q0.y + qi.z * q0.z + qi.w * q0.w;
                float sg = (i > 0 && dq < 0.f) ? -wi : wi;
                q.x += sg * qi.x; q.y += sg * qi.y; q.z += sg * qi.z; q.w += sg * qi.w;
            }
            float L = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            const float4 c2 = a.copies[4 * (size_t)e0 + 2], c3 = a.copies[4 * (size_t)e0 + 3];
            o0 = make_float4(xs.x + h * v.x, xs.y + h * v.y, xs.z + h * v.z, x0.w);
            o1 = make_float4(q.x / L, q.y / L, q.z / L, q.w / L);
            o2 = make_float4(v.x, v.y, v.z, c2.w);
            o3 = make_float4(w.x, w.y, w.z, c3.w);
        }
        bool finite = isfinite(o0.x) && isfinite(o0.y) && isfinite(o0.z) && isfinite(o1.x) &&
                      isfinite(o1.y) && isfinite(o1.z) && isfinite(o1.w) && isfinite(o2.x) &&
                      isfinite(o2.y) && isfinite(o2.z) && isfinite(o3.x) && isfinite(o3.y) &&
                      isfinite(o3.z);
        if (!finite) atomicCAS(a.status, DEV_OK, DEV_ERR_NONFINITE);
        a.st_out[4 * b] = o0; a.st_out[4 * b + 1] = o1; a.st_out[4 * b + 2] = o2; a.st_out[4 * b + 3] = o3;
    }
}

constexpr int JERR_THREADS = 512;

// one CTA: thread t sums the joints t, t + T, ... in FP64, then a fixed tree
// over the threads, so the sum does not depend on scheduling
__global__ void __launch_bounds__(JERR_THREADS)
k_joint_error(const int2 *jab, const float4 *janc, const float4 *st, int nj, double *out) {
    __shared__ double s_sum[JERR_THREADS];
    __shared__ float s_max[JERR_THREADS];
    double sum = 0.0;
    float mx = 0.f;
    for (int j = threadIdx.x; j < nj; j += JERR_THREADS) {
        const int2 ab = jab[j];
        const float4 anA = janc[2 * j], anB = janc[2 * j + 1];
        float3 xA, xB, rA = make_float3(0.f, 0.f, 0.f), rB = rA;
        if (ab.x >= 0) {
            const float4 x = st[4 * ab.x];
            xA = make_float3(x.x, x.y, x.z);
            rA = quat_rotate(st[4 * ab.x + 1], make_float3(anA.x, anA.y, anA.z));
        } else {
            xA = make_float3(anA.x, anA.y, anA.z);
        }
        if (ab.y >= 0) {
            const float4 x = st[4 * ab.y];
            xB = make_float3(x.x, x.y, x.z);
            rB = quat_rotate(st[4 * ab.y + 1], make_float3(anB.x, anB.y, anB.z));
        } else {
            xB = make_float3(anB.x, anB.y, anB.z);
        }
        // nearby large coordinates subtracted first, as in the joint rows
        const float dx = (xB.x - xA.x) + (rB.x - rA.x), dy = (xB.y - xA.y) + (rB.y - rA.y),
                    dz = (xB.z - xA.z) + (rB.z - rA.z);
        const float g = sqrtf(dx * dx + dy * dy + dz * dz);
        sum += (double)g;
        mx = fmaxf(mx, g);
    }
    s_sum[threadIdx.x] = sum;
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int w = JERR_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
            s_max[threadIdx.x] = fmaxf(s_max[threadIdx.x], s_max[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s_sum[0]; out[1] = (double)s_max[0]; }
}

__global__ void k_pack(const float *in, const float *radius, const float *im, int n, float4 *st) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const float *s = in + 13 * (size_t)b;
        float r = radius[b], m = im[b];
        float ii = m > 0.f ? m / (0.4f * r * r) : 0.f;   // solid sphere I = 2/5 m r^2
        st[4 * b] = make_float4(s[0], s[1], s[2], r);
        st[4 * b + 1] = make_float4(s[3], s[4], s[5], s[6]);
        st[4 * b + 2] = make_float4(s[7], s[8], s[9], m);
        st[4 * b + 3] = make_float4(s[10], s[11], s[12], ii);
    }
}

__global__ void k_unpack(const float4 *st, int n, float *out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        float *o = out + 13 * (size_t)b;
        float4 x = st[4 * b], q = st[4 * b + 1], v = st[4 * b + 2], w = st[4 * b + 3];
        o[0] = x.x; o[1] = x.y; o[2] = x.z;
        o[3] = q.x; o[4] = q.y; o[5] = q.z; o[6] = q.w;
        o[7] = v.x; o[8] = v.y; o[9] = v.z;
        o[10] = w.x; o[11] = w.y; o[12] = w.z;
    }
}

}  // namespace

void launch_geo_sources(const GeoArgs &a, cudaStream_t s) {
    k_geo_sources<<<grid1d(a.n, 256), 256, 0, s>>>(a);
    note_launch();
    k_geo_mark<<<1, 1, 0, s>>>(a.qctl, 1);
    note_launch();
    CK(cudaGetLastError());
}

void launch_geo_level(const GeoArgs &a, int level, cudaStream_t s) {
    k_geo_level<<<152 * 8, 256, 0, s>>>(a, level);
    note_launch();
    k_geo_mark<<<1, 1, 0, s>>>(a.qctl, level + 1);
    note_launch();
    CK(cudaGetLastError());
}

void launch_joint_error(const int2 *jab, const float4 *janc, const float4 *st, int nj, double *out,
                        cudaStream_t s) {
    k_joint_error<<<1, JERR_THREADS, 0, s>>>(jab, janc, st, nj, out);
    note_launch();
    CK(cudaGetLastError());
}

void launch_blend(const BlendArgs &a, cudaStream_t s) {
    k_blend<<<grid1d(a.n, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

void launch_pack_state(const float *in13, const float *radius, const float *im, int n, float4 *st,
                       cudaStream_t s) {
    k_pack<<<grid1d(n, 256), 256, 0, s>>>(in13, radius, im, n, st);
    note_launch();
    CK(cudaGetLastError());
}

void launch_unpack_state(const float4 *st, int n, float *out13, cudaStream_t s) {
    k_unpack<<<grid1d(n, 256), 256, 0, s>>>(st, n, out13);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
