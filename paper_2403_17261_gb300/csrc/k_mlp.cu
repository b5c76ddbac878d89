// k_mlp.cu -- the learned warm start (not part of the paper's method): per
// contact features, a 12-64-64-3 ReLU network that proposes the contact's
// three impulses, the log of (features, converged impulses) the solver
// produces, and the network's training.
//
// Features of a (worker, contact) pair, from the blended state at the start
// of the step (before gravity), with g_ref = max(|g|, 1) and
// s = g_ref h / (im_A + im_B) over the dynamic ends:
//   0-2  J v along n, t1, t2 (static ends have v = 0) / (g_ref h)
//   3    penetration max(-phi, 0) / (g_ref h^2)
//   4-6  the previous-step impulses the plain warm start applies / s
//   7-8  inverse masses of the two ends (0 when static or a plane)
//   9-10 their degrees in G^t / 8
//   11   min over the dynamic ends of the BFS distance to O (capped at 8) / 8
// The network's outputs are impulses / s, y = x[4:7] + W3^T relu(W2^T
// relu(W1^T x + b1) + b2) + b3: the layers correct the previous-step impulses
// (features 4-6, added in FP32).  A warm start takes s y, keeps the normal
// impulse non-negative and clamps each friction impulse to mu times it.
//
// Inference runs on the 5th-generation tensor cores: tcgen05.mma with BF16
// operands in shared memory and FP32 accumulators in tensor memory, 128 pairs
// per CTA at a time (one MMA for layer 1, four K-steps each for layers 2 and
// 3); the epilogue of each layer reads its accumulator rows from tensor
// memory (tcgen05.ld), adds the bias, applies the ReLU and writes the next
// layer's BF16 operand to shared memory.  Training runs on the tensor cores
// too, with the same arithmetic (operands rounded to BF16, products exact,
// FP32 sums): the forward and backward passes of 128 samples per CTA as five
// products, the weight gradients of 128 samples per CTA as three products
// with the samples as K, summed over blocks in block order (deterministic),
// and Adam on FP32 master parameters.
#include <cuda_bf16.h>

#include <algorithm>
#include <stdexcept>

#include "common.cuh"
#include "kernels.cuh"

namespace ovl {

namespace {

// parameter vector (C ABI layout)
constexpr int OFF_W1 = 0, OFF_B1 = 768, OFF_W2 = 832, OFF_B2 = 4928, OFF_W3 = 4992, OFF_B3 = 5184;
static_assert(OFF_B3 + 3 == MLP_N_PARAMS, "parameter layout");
// packed inference weights (32-bit words): the MMAs' B operands in the
// K-major, unswizzled tensor-core layout (below) -- W1^T [64 x 16] (inputs
// 12-15 zero), W2^T [64 x 64], W3^T [16 x 64] (outputs 3-15 zero) -- then
// FP32 biases b1 [64], b2 [64], b3 [16] (zero-padded)
constexpr int PK_W1 = 0, PK_W2 = 512, PK_W3 = 2560, PK_B1 = 3072, PK_B2 = 3136, PK_B3 = 3200;
static_assert(PK_B3 + 16 == MLP_PK_WORDS, "packed layout");
// activation rows of the training pass
constexpr int A_X = 0, A_H1 = 16, A_H2 = 80, A_DZ1 = 144, A_DZ2 = 208, A_DY = 272;
static_assert(A_DY + 4 == MLP_ACT_STRIDE, "activation layout");

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}

// ---- tensor-core operands and instructions (tcgen05) --------------------------
// A K-major operand with K columns, unswizzled: 8 x 8 core matrices (8 rows of
// 16 B, 128 B each), the core matrices of one 8-row group adjacent along K
// (leading byte offset 128 B), the 8-row groups K * 16 B apart (stride byte
// offset).  Byte offset of element (row r, column k):
__host__ __device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed 0b001 at
// 46-48, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (uint64_t)((lbo >> 4) & 0x3FFFu) << 16 |
           (uint64_t)((sbo >> 4) & 0x3FFFu) << 32 | (uint64_t)1 << 46;
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A B^T for M = 128 rows, one K = 16 step; issued by one thread
__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc ? 1u : 0u) : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

// waits for phase `parity` of the mbarrier; false after the iteration limit
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// this thread's accumulator row (TMEM lane = row), 16 columns from column col
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---- depth to O ------------------------------------------------------------

__global__ void k_depth_init(const uint64_t *mask, int n, uint8_t *depth) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x)
        depth[b] = __popcll(mask[b]) >= 2 ? 0 : MLP_DEPTH_CAP;
}

// Vertices at level L-1 mark their unreached neighbours with L.  Only the
// value L is written during a level, so concurrent writes agree.
__global__ void k_depth_level(const int *row_ptr, const int *col, int n, uint8_t *depth, int L) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (depth[u] != L - 1) continue;
        for (int k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            const int v = col[k];
            if (depth[v] == MLP_DEPTH_CAP) depth[v] = (uint8_t)L;
        }
    }
}

// ---- features ----------------------------------------------------------------

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__global__ void k_features(FeatArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.np; k += gridDim.x * blockDim.x) {
        const int i = a.ps_cons[k], p = a.ps_part[k];
        const uint64_t key = a.p_key[k];
        int lo = a.ws.ws_pstart[p], hi = a.ws.ws_pstart[p + 1];
        const int end = hi;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.ws.ws_key[mid] < key) lo = mid + 1; else hi = mid;
        }
        const bool found = lo < end && a.ws.ws_key[lo] == key;
        float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0, o2 = o0;
        float4 meta = make_float4(found ? 1.f : 0.f, 0.f, 0.f, 0.f);
        const bool contact = i < a.nc;
        if (contact) {
            const int2 ab = a.c_ab[i];
            const float4 nphi = a.c_n[i];
            const float3 n = f3(nphi), t1 = f3(a.c_t1[i]), t2 = cross(n, t1);
            float3 pa = make_float3(0.f, 0.f, 0.f), pb = pa;
            const float4 va = a.st[4 * ab.x + 2];
            const float ima = va.w;   // 0 for a static body
            if (ima > 0.f) {
                const float ra = a.st[4 * ab.x].w;
                const float3 w = f3(a.st[4 * ab.x + 3]);
                const float3 wr = cross(w, make_float3(ra * n.x, ra * n.y, ra * n.z));
                pa = make_float3(va.x + wr.x, va.y + wr.y, va.z + wr.z);
            }
            float imb = 0.f;
            if (ab.y < a.n) {
                const float4 vb = a.st[4 * ab.y + 2];
                if (vb.w > 0.f) {
                    imb = vb.w;
                    const float rb = a.st[4 * ab.y].w;
                    const float3 w = f3(a.st[4 * ab.y + 3]);
                    const float3 wr = cross(w, make_float3(-rb * n.x, -rb * n.y, -rb * n.z));
                    pb = make_float3(vb.x + wr.x, vb.y + wr.y, vb.z + wr.z);
                }
            }
            const float3 rel = make_float3(pb.x - pa.x, pb.y - pa.y, pb.z - pa.z);
            const int scene = a.part_scene[p];
            const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[scene];
            const float gh = a.g_ref * h;
            const float scale = gh / (ima + imb);
            float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
            if (found) {
                const float4 v = a.ws.ws_lam[lo];
                l = make_float4(v.x * a.ws.factor, v.y * a.ws.factor, v.z * a.ws.factor, 0.f);
            }
            const bool dyn_b = imb > 0.f;
            int d = MLP_DEPTH_CAP;
            if (ima > 0.f) d = min(d, (int)a.depth[ab.x]);
            if (dyn_b) d = min(d, (int)a.depth[ab.y]);
            const float dga = ima > 0.f ? (float)(a.row_ptr[ab.x + 1] - a.row_ptr[ab.x]) * 0.125f : 0.f;
            const float dgb = dyn_b ? (float)(a.row_ptr[ab.y + 1] - a.row_ptr[ab.y]) * 0.125f : 0.f;
            o0 = make_float4(dot(n, rel) / gh, dot(t1, rel) / gh, dot(t2, rel) / gh,
                             fmaxf(-nphi.w, 0.f) / (gh * h));
            o1 = make_float4(l.x / scale, l.y / scale, l.z / scale, ima);
            o2 = make_float4(imb, dga, dgb, (float)d / (float)MLP_DEPTH_CAP);
            meta = make_float4(found ? 1.f : 0.f, scale, a.scene_mu[scene], 1.f);
        }
        a.feat[4 * (size_t)k] = o0;
        a.feat[4 * (size_t)k + 1] = o1;
        a.feat[4 * (size_t)k + 2] = o2;
        a.feat[4 * (size_t)k + 3] = meta;
        a.is_contact[k] = contact ? 1 : 0;
    }
}

// ---- inference ---------------------------------------------------------------

__global__ void k_mlp_pack(const float *th, uint32_t *pk) {
    uint8_t *w = reinterpret_cast<uint8_t *>(pk);
    auto put = [&](int word0, int r, int k, int K, float v) {
        *reinterpret_cast<__nv_bfloat16 *>(w + 4 * word0 + kmajor_off(r, k, K)) = __float2bfloat16_rn(v);
    };
    for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {    // W1^T: row = output, column = input
        const int n = e / 16, k = e % 16;
        put(PK_W1, n, k, 16, k < 12 ? th[OFF_W1 + k * 64 + n] : 0.f);
    }
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int n = e / 64, k = e % 64;
        put(PK_W2, n, k, 64, th[OFF_W2 + k * 64 + n]);
    }
    for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
        const int n = e / 64, k = e % 64;
        put(PK_W3, n, k, 64, n < 3 ? th[OFF_W3 + k * 3 + n] : 0.f);
    }
    float *bias = reinterpret_cast<float *>(pk);
    for (int e = threadIdx.x; e < 64; e += blockDim.x) {
        bias[PK_B1 + e] = th[OFF_B1 + e];
        bias[PK_B2 + e] = th[OFF_B2 + e];
    }
    for (int e = threadIdx.x; e < 16; e += blockDim.x) bias[PK_B3 + e] = e < 3 ? th[OFF_B3 + e] : 0.f;
}

template <int MODE>
__device__ __forceinline__ void infer_store(int r, int n, float y0, float y1, float y2,
                                            const float4 *feat, float4 *lam0, float *y3) {
    if (r >= n) return;
    // skip connection: features 4-6 (previous impulses / s), in FP32
    const float4 f1 = feat[4 * (size_t)r + 1];
    y0 += f1.x; y1 += f1.y; y2 += f1.z;
    if (MODE == 0) {
        y3[3 * (size_t)r] = y0; y3[3 * (size_t)r + 1] = y1; y3[3 * (size_t)r + 2] = y2;
        return;
    }
    const float4 meta = feat[4 * (size_t)r + 3];   // found, scale, mu, contact
    if (meta.w == 0.f) return;                    // joints keep the previous impulses
    if (MODE == 2 && meta.x != 0.f) return;       // contacts seen last step keep them too
    const float ln = fmaxf(meta.y * y0, 0.f), lim = meta.z * ln;
    lam0[r] = make_float4(ln, fminf(fmaxf(meta.y * y1, -lim), lim),
                          fminf(fmaxf(meta.y * y2, -lim), lim), 0.f);
}

// One CTA of 128 threads holds the weights in shared memory and takes tiles
// of 128 pairs in turn; thread t owns row t of a tile (TMEM lane t).  Per
// tile: X (12 features + 4 zero columns, BF16) -> D1 = X W1 (one MMA) ->
// H = relu(D1 + b1) -> D2 = H W2 (four K-steps) -> H = relu(D2 + b2) -> D3
// = H W3 (N = 16, four K-steps) -> y = D3 + b3.  Accumulators: D1 and D3 in
// TMEM columns 0-63 (D3 in 0-15), D2 in 64-127.  Every wait on an MMA is
// bounded; a wait that gives up sets the device status, and the CTA stops
// taking tiles, waits once more and frees its tensor memory.
constexpr int INFER_THREADS = 128, INFER_COLS = 128;

template <int MODE>
__global__ void __launch_bounds__(INFER_THREADS) k_mlp_infer(const uint32_t *pk, const float4 *feat, int n,
                                                            float4 *lam0, float *y3, int *status) {
    __shared__ __align__(1024) uint8_t sw1[64 * 16 * 2];
    __shared__ __align__(1024) uint8_t sw2[64 * 64 * 2];
    __shared__ __align__(1024) uint8_t sw3[16 * 64 * 2];
    __shared__ __align__(1024) uint8_t sx[128 * 16 * 2];
    __shared__ __align__(1024) uint8_t sh[128 * 64 * 2];
    __shared__ float sb[64 + 64 + 16];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    {
        const uint32_t *src = pk;
        for (int i = tid; i < 512; i += INFER_THREADS) reinterpret_cast<uint32_t *>(sw1)[i] = src[PK_W1 + i];
        for (int i = tid; i < 2048; i += INFER_THREADS) reinterpret_cast<uint32_t *>(sw2)[i] = src[PK_W2 + i];
        for (int i = tid; i < 512; i += INFER_THREADS) reinterpret_cast<uint32_t *>(sw3)[i] = src[PK_W3 + i];
        const float *b = reinterpret_cast<const float *>(pk);
        for (int i = tid; i < 144; i += INFER_THREADS) sb[i] = b[PK_B1 + i];
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "n"(INFER_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 rows
    const uint32_t ax = (uint32_t)__cvta_generic_to_shared(sx), ah = (uint32_t)__cvta_generic_to_shared(sh);
    const uint32_t b1a = (uint32_t)__cvta_generic_to_shared(sw1), b2a = (uint32_t)__cvta_generic_to_shared(sw2),
                   b3a = (uint32_t)__cvta_generic_to_shared(sw3);
    uint32_t phase = 0;
    bool ok = true;
    const int tiles = (n + 127) >> 7;
    // this thread's features of its row of a tile (zeros past the end); the
    // next tile's are loaded while the current tile's MMAs run
    auto load_row = [&](int t, float *x) {
        const int rr = 128 * t + tid;
#pragma unroll
        for (int k = 0; k < 12; ++k) x[k] = 0.f;
        if (t < tiles && rr < n) {
            const float4 *f = feat + 4 * (size_t)rr;
            const float4 a = f[0], b = f[1], c = f[2];
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y;
            x[6] = b.z; x[7] = b.w; x[8] = c.x; x[9] = c.y; x[10] = c.z; x[11] = c.w;
        }
    };
    float xn[12];
    load_row(blockIdx.x, xn);
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int r = 128 * tile + tid;
        // layer-1 operand: this thread's row, features 0-11 and four zeros
        {
            float x[16];
#pragma unroll
            for (int k = 0; k < 12; ++k) x[k] = xn[k];
            x[12] = x[13] = x[14] = x[15] = 0.f;
            uint32_t q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = pack_bf16(x[2 * k], x[2 * k + 1]);
            *reinterpret_cast<uint4 *>(sx + kmajor_off(tid, 0, 16)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(sx + kmajor_off(tid, 8, 16)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
            umma_f16(tmem, umma_desc(ax, 128, 16 * 16), umma_desc(b1a, 128, 16 * 16), umma_idesc(128, 64), false);
            umma_commit(mb);
        }
        load_row(tile + gridDim.x, xn);
        ok = __syncthreads_and(mbar_wait(mb, phase));   // the same decision in every thread
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
        // H = relu(D + b) as this row of the next operand, twice (layers 1, 2)
#pragma unroll 1
        for (int layer = 0; layer < 2; ++layer) {
            const uint32_t dcol = layer == 0 ? 0u : 64u;
            const float *bias = sb + 64 * layer;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float v[16];
                tmem_ld16(lane_base + dcol + c0, v);
                uint32_t q[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    q[k] = pack_bf16(fmaxf(v[2 * k] + bias[c0 + 2 * k], 0.f), fmaxf(v[2 * k + 1] + bias[c0 + 2 * k + 1], 0.f));
                *reinterpret_cast<uint4 *>(sh + kmajor_off(tid, c0, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
                *reinterpret_cast<uint4 *>(sh + kmajor_off(tid, c0 + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_sync();
            if (tid == 0) {
                // layer 2 into D2 (columns 64-127); layer 3 (N = 16) into columns 0-15
                const uint32_t d = layer == 0 ? tmem + 64u : tmem;
                const uint32_t bop = layer == 0 ? b2a : b3a;
                const uint32_t idesc = layer == 0 ? umma_idesc(128, 64) : umma_idesc(128, 16);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    umma_f16(d, umma_desc(ah + 256u * ks, 128, 64 * 16), umma_desc(bop + 256u * ks, 128, 64 * 16), idesc, ks > 0);
                umma_commit(mb);
            }
            ok = __syncthreads_and(mbar_wait(mb, phase));
            phase ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok) break;
        }
        if (!ok) break;
        float o[16];
        tmem_ld16(lane_base, o);
        const float *b3 = sb + 128;
        infer_store<MODE>(r, n, o[0] + b3[0], o[1] + b3[1], o[2] + b3[2], feat, lam0, y3);
        tc_sync();   // every row read out before the next tile's MMAs reuse the operands and columns
    }
    if (!ok) {
        if (tid == 0) atomicCAS(status, DEV_OK, DEV_ERR_TIMEOUT);
        mbar_wait(mb, phase ^ 1u);   // the product that was not seen to finish, once more (bounded)
    }
    tc_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(INFER_COLS) : "memory");
}

// ---- log -----------------------------------------------------------------------

__global__ void k_log_append(const float4 *feat, const float4 *lam, const int *pos, int np,
                             float *log_feat, float *log_targ, long long base, long long cap) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const float4 meta = feat[4 * (size_t)k + 3];
        if (meta.w == 0.f) continue;
        const long long row = base + pos[k];
        if (row >= cap) continue;
        const float4 f0 = feat[4 * (size_t)k], f1 = feat[4 * (size_t)k + 1], f2 = feat[4 * (size_t)k + 2];
        float *o = log_feat + 12 * row;
        o[0] = f0.x; o[1] = f0.y; o[2] = f0.z; o[3] = f0.w;
        o[4] = f1.x; o[5] = f1.y; o[6] = f1.z; o[7] = f1.w;
        o[8] = f2.x; o[9] = f2.y; o[10] = f2.z; o[11] = f2.w;
        const float4 l = lam[k];
        float *tg = log_targ + 3 * row;
        tg[0] = l.x / meta.y; tg[1] = l.y / meta.y; tg[2] = l.z / meta.y;
    }
}

// ---- training --------------------------------------------------------------------

constexpr int WGRAD_CHUNK = 128;   // samples of one gradient block (one tensor-core K = 128 product)

__device__ __forceinline__ long long sample_row(const TrainArgs &a, long long step, int j) {
    if (a.sampling == 0) return a.first + (long long)(((unsigned long long)step * a.batch + j) % (unsigned long long)a.count);
    const uint64_t z = mix64(a.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(step * (long long)a.batch + j + 1));
    return a.first + (long long)(z % (uint64_t)a.count);
}

// Forward, loss and the backward pass down to the pre-activation gradients
// of one tile of 128 samples per CTA, on the tensor cores; thread t owns
// sample t of the tile (TMEM lane t).  Five products, each M = 128 with BF16
// operands in shared memory and FP32 accumulators in tensor memory:
//   D1 = X W1 (K 16), D2 = H1 W2 (K 64), D3 = H2 W3 (N 16, K 64),
//   T2 = dY W3^T (K 16, dY in columns 0-2), T1 = dZ2 W2^T (K 64),
// with h1 = bf16(relu(D1 + b1)), h2 = bf16(relu(D2 + b2)), y = (D3 + b3) +
// x[4..6] (the skip connection in FP32), dy = bf16(2 (y - t) / (3 B)),
// dz2 = bf16(T2) where h2 > 0, dz1 = bf16(T1) where h1 > 0.  Every operand
// of a product is BF16 (the products exact) and the sums FP32.  The B
// operands are built from the FP32 parameters by every CTA.  Accumulators:
// D1 and then T1 in TMEM columns 0-63, D2 in 64-127, D3 in 128-143, T2 in
// 192-255.  Waits on the MMAs are bounded; one that gives up sets the device
// status, and the CTA waits once more and frees its tensor memory.
constexpr int TRAIN_TILE = 128, TRAIN_COLS = 256;
constexpr int TF_X = 0, TF_H1 = TF_X + 128 * 16 * 2, TF_H2 = TF_H1 + 128 * 64 * 2, TF_DY = TF_H2 + 128 * 64 * 2,
              TF_DZ2 = TF_DY + 128 * 16 * 2, TF_B1 = TF_DZ2 + 128 * 64 * 2, TF_B2 = TF_B1 + 64 * 16 * 2,
              TF_B3 = TF_B2 + 64 * 64 * 2, TF_B4 = TF_B3 + 16 * 64 * 2, TF_B5 = TF_B4 + 64 * 16 * 2,
              TF_SMEM = TF_B5 + 64 * 64 * 2;
// two CTAs per SM at most: each holds half of the SM's 512 tensor-memory
// columns, and a third would wait in tcgen05.alloc
static_assert(3 * (TF_SMEM + 2048) > 228 * 1024 && 2 * (TF_SMEM + 2048) <= 227 * 1024, "two CTAs per SM");

// one row (K columns) of a K-major BF16 operand from FP32 values
template <int K>
__device__ __forceinline__ void put_row(uint8_t *op, int r, const float *v) {
#pragma unroll
    for (int c = 0; c < K; c += 8) {
        uint4 q;
        q.x = pack_bf16(v[c], v[c + 1]); q.y = pack_bf16(v[c + 2], v[c + 3]);
        q.z = pack_bf16(v[c + 4], v[c + 5]); q.w = pack_bf16(v[c + 6], v[c + 7]);
        *reinterpret_cast<uint4 *>(op + kmajor_off(r, c, K)) = q;
    }
}

__global__ void __launch_bounds__(TRAIN_TILE) k_train_fwd(TrainArgs a) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ float sb[64 + 64 + 4];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    // B operands from the parameters: row n, column k
    {
        const float *th = a.theta;
        auto put = [&](int off, int r, int k, int K, float v) {
            *reinterpret_cast<__nv_bfloat16 *>(tsm + off + kmajor_off(r, k, K)) = __float2bfloat16_rn(v);
        };
        for (int e = tid; e < 64 * 16; e += TRAIN_TILE) {
            const int n = e / 16, k = e % 16;
            put(TF_B1, n, k, 16, k < 12 ? th[OFF_W1 + k * 64 + n] : 0.f);        // W1^T
            put(TF_B4, n, k, 16, k < 3 ? th[OFF_W3 + n * 3 + k] : 0.f);          // (W3^T)^T = W3
        }
        for (int e = tid; e < 64 * 64; e += TRAIN_TILE) {
            const int n = e / 64, k = e % 64;
            put(TF_B2, n, k, 64, th[OFF_W2 + k * 64 + n]);                       // W2^T
            put(TF_B5, n, k, 64, th[OFF_W2 + n * 64 + k]);                       // (W2^T)^T = W2
        }
        for (int e = tid; e < 16 * 64; e += TRAIN_TILE) {
            const int n = e / 64, k = e % 64;
            put(TF_B3, n, k, 64, n < 3 ? th[OFF_W3 + k * 3 + n] : 0.f);          // W3^T
        }
        for (int e = tid; e < 64; e += TRAIN_TILE) { sb[e] = th[OFF_B1 + e]; sb[64 + e] = th[OFF_B2 + e]; }
        if (tid < 4) sb[128 + tid] = tid < 3 ? th[OFF_B3 + tid] : 0.f;
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(dst), "n"(TRAIN_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // this thread's sample: features (rounded to BF16 for the product, FP32
    // for the skip connection) and targets
    const long long step = a.step_dev ? *a.step_dev : a.step;
    const int j = blockIdx.x * TRAIN_TILE + tid;
    const bool valid = j < a.batch;
    float xraw[12], targ[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 12; ++k) xraw[k] = 0.f;
    long long r = 0;
    if (valid) {
        r = sample_row(a, step, j);
        const float4 *f = reinterpret_cast<const float4 *>(a.log_feat + 12 * r);
        const float4 f0 = f[0], f1 = f[1], f2 = f[2];
        xraw[0] = f0.x; xraw[1] = f0.y; xraw[2] = f0.z; xraw[3] = f0.w; xraw[4] = f1.x; xraw[5] = f1.y;
        xraw[6] = f1.z; xraw[7] = f1.w; xraw[8] = f2.x; xraw[9] = f2.y; xraw[10] = f2.z; xraw[11] = f2.w;
        targ[0] = a.log_targ[3 * r]; targ[1] = a.log_targ[3 * r + 1]; targ[2] = a.log_targ[3 * r + 2];
    }
    float *act = a.act + (size_t)(valid ? j : 0) * MLP_ACT_STRIDE;
    const bool wr = valid && a.backward;
    {
        float x[16];
#pragma unroll
        for (int k = 0; k < 12; ++k) x[k] = bf16r(xraw[k]);
        x[12] = x[13] = x[14] = x[15] = 0.f;
        put_row<16>(tsm + TF_X, tid, x);
        if (wr)
#pragma unroll
            for (int c = 0; c < 16; c += 4) *reinterpret_cast<float4 *>(act + A_X + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tsm);
    uint32_t phase = 0;
    bool ok = true;
    // one product (ks K-steps of 16) into columns dcol, then the wait
    auto mma = [&](uint32_t dcol, int aoff, int boff, int K, int N) {
        if (tid == 0) {
            const uint32_t sbo = (uint32_t)K * 16u;
            for (int ks = 0; ks < K / 16; ++ks)
                umma_f16(tmem + dcol, umma_desc(base + aoff + 256u * ks, 128, sbo),
                         umma_desc(base + boff + 256u * ks, 128, sbo), umma_idesc(128, N), ks > 0);
            umma_commit(mb);
        }
        ok = __syncthreads_and(mbar_wait(mb, phase));
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };
    uint64_t m1 = 0, m2 = 0;   // h1 > 0, h2 > 0 per hidden unit
    // h = bf16(relu(D + b)) into the next operand (and the activation row)
    auto hidden = [&](uint32_t dcol, const float *bias, int opoff, int aoff_act, uint64_t &mask) {
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + dcol + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = bf16r(fmaxf(v[i] + bias[c0 + i], 0.f));
                if (v[i] > 0.f) mask |= 1ull << (c0 + i);
            }
            uint8_t *op = tsm + opoff;
#pragma unroll
            for (int c = 0; c < 16; c += 8) {
                uint4 q;
                q.x = pack_bf16(v[c], v[c + 1]); q.y = pack_bf16(v[c + 2], v[c + 3]);
                q.z = pack_bf16(v[c + 4], v[c + 5]); q.w = pack_bf16(v[c + 6], v[c + 7]);
                *reinterpret_cast<uint4 *>(op + kmajor_off(tid, c0 + c, 64)) = q;
            }
            if (wr)
#pragma unroll
                for (int c = 0; c < 16; c += 4)
                    *reinterpret_cast<float4 *>(act + aoff_act + c0 + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
    };
    // delta = bf16(T) where the unit is active, into the activation row (and
    // an operand when opoff >= 0)
    auto delta = [&](uint32_t dcol, uint64_t mask, int opoff, int aoff_act) {
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + dcol + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = (mask >> (c0 + i) & 1ull) ? bf16r(v[i]) : 0.f;
            if (opoff >= 0) {
                uint8_t *op = tsm + opoff;
#pragma unroll
                for (int c = 0; c < 16; c += 8) {
                    uint4 q;
                    q.x = pack_bf16(v[c], v[c + 1]); q.y = pack_bf16(v[c + 2], v[c + 3]);
                    q.z = pack_bf16(v[c + 4], v[c + 5]); q.w = pack_bf16(v[c + 6], v[c + 7]);
                    *reinterpret_cast<uint4 *>(op + kmajor_off(tid, c0 + c, 64)) = q;
                }
            }
            if (wr)
#pragma unroll
                for (int c = 0; c < 16; c += 4)
                    *reinterpret_cast<float4 *>(act + aoff_act + c0 + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
    };
    mma(0u, TF_X, TF_B1, 16, 64);
    if (ok) { hidden(0u, sb, TF_H1, A_H1, m1); mma(64u, TF_H1, TF_B2, 64, 64); }
    if (ok) { hidden(64u, sb + 64, TF_H2, A_H2, m2); mma(128u, TF_H2, TF_B3, 64, 16); }
    if (ok) {
        float o[16];
        tmem_ld16(lane_base + 128u, o);
        float dy[16], loss = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) dy[k] = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float y = (o[k] + sb[128 + k]) + xraw[4 + k];
            const float d = y - targ[k];
            loss += d * d;
            dy[k] = bf16r(2.f * d / (3.f * (float)a.batch));
        }
        if (valid) a.sample_loss[j] = loss;
        if (wr) *reinterpret_cast<float4 *>(act + A_DY) = make_float4(dy[0], dy[1], dy[2], 0.f);
        if (a.backward) {
            put_row<16>(tsm + TF_DY, tid, dy);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_sync();
            mma(192u, TF_DY, TF_B4, 16, 64);
            if (ok) { delta(192u, m2, TF_DZ2, A_DZ2); mma(0u, TF_DZ2, TF_B5, 64, 64); }
            if (ok) delta(0u, m1, -1, A_DZ1);
        }
    }
    if (!ok) {
        if (tid == 0) atomicCAS(a.status, DEV_OK, DEV_ERR_TIMEOUT);
        mbar_wait(mb, phase ^ 1u);   // the product that was not seen to finish, once more (bounded)
    }
    tc_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(TRAIN_COLS) : "memory");
}

// Block-partial gradients over the WGRAD_CHUNK = 128 samples of one CTA, on
// the tensor cores: every weight gradient is a sum over samples of (operand
// A) x (operand B) of the activation rows (all BF16 values, so the products
// are exact), i.e. a GEMM with the samples as K:
//   dW1 = X^T dZ1 (12 x 64), dW2 = H1^T dZ2 (64 x 64), dW3 = H2^T dY (64 x 3),
// and a bias gradient is the same sum with A = 1.  Each GEMM is one M = 128
// tcgen05 product over K = 128 samples (eight K-steps): A holds the
// transposed activations in its first rows and a row of ones after them (its
// accumulator row is the bias gradient), B the transposed deltas; thread s
// writes sample s's column of every operand.  Accumulators: dW1 in TMEM
// columns 0-63, dW2 in 64-127, dW3 in 128-143.  Slot MLP_N_PARAMS of a
// block's partials holds its loss sum.
constexpr int WG_A_BYTES = 128 * WGRAD_CHUNK * 2, WG_B_BYTES = 64 * WGRAD_CHUNK * 2, WG_B3_BYTES = 16 * WGRAD_CHUNK * 2;
constexpr int WG_SMEM = 3 * WG_A_BYTES + 2 * WG_B_BYTES + WG_B3_BYTES;

__global__ void __launch_bounds__(WGRAD_CHUNK) k_train_wgrad(TrainArgs a) {
    extern __shared__ __align__(1024) uint8_t wsm[];
    uint8_t *A1 = wsm, *A2 = A1 + WG_A_BYTES, *A3 = A2 + WG_A_BYTES;
    uint8_t *B1 = A3 + WG_A_BYTES, *B2 = B1 + WG_B_BYTES, *B3 = B2 + WG_B_BYTES;
    __shared__ float lsum[WGRAD_CHUNK];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int s0 = blockIdx.x * WGRAD_CHUNK, cnt = min(WGRAD_CHUNK, a.batch - s0);
    for (int i = tid; i < WG_SMEM / 16; i += WGRAD_CHUNK) reinterpret_cast<uint4 *>(wsm)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // this sample's column of every operand (zeros past the batch)
    {
        const bool valid = tid < cnt;
        const float *r = a.act + (size_t)(s0 + (valid ? tid : 0)) * MLP_ACT_STRIDE;
        auto put = [&](uint8_t *op, int row, float v) {
            *reinterpret_cast<__nv_bfloat16 *>(op + kmajor_off(row, tid, WGRAD_CHUNK)) = __float2bfloat16_rn(valid ? v : 0.f);
        };
        for (int k = 0; k < 12; ++k) put(A1, k, r[A_X + k]);
        put(A1, 12, 1.f);
        for (int k = 0; k < 64; ++k) {
            put(A2, k, r[A_H1 + k]);
            put(A3, k, r[A_H2 + k]);
            put(B1, k, r[A_DZ1 + k]);
            put(B2, k, r[A_DZ2 + k]);
        }
        put(A2, 64, 1.f);
        put(A3, 64, 1.f);
        for (int j = 0; j < 3; ++j) put(B3, j, r[A_DY + j]);
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint32_t sbo = WGRAD_CHUNK * 16;
        const uint32_t a1 = (uint32_t)__cvta_generic_to_shared(A1), a2 = (uint32_t)__cvta_generic_to_shared(A2),
                       a3 = (uint32_t)__cvta_generic_to_shared(A3), b1 = (uint32_t)__cvta_generic_to_shared(B1),
                       b2 = (uint32_t)__cvta_generic_to_shared(B2), b3 = (uint32_t)__cvta_generic_to_shared(B3);
#pragma unroll 1
        for (int ks = 0; ks < WGRAD_CHUNK / 16; ++ks) {
            const uint32_t o = 256u * ks;
            umma_f16(tmem, umma_desc(a1 + o, 128, sbo), umma_desc(b1 + o, 128, sbo), umma_idesc(128, 64), ks > 0);
            umma_f16(tmem + 64u, umma_desc(a2 + o, 128, sbo), umma_desc(b2 + o, 128, sbo), umma_idesc(128, 64), ks > 0);
            umma_f16(tmem + 128u, umma_desc(a3 + o, 128, sbo), umma_desc(b3 + o, 128, sbo), umma_idesc(128, 16), ks > 0);
        }
        umma_commit(mb);
    }
    const bool ok = __syncthreads_and(mbar_wait(mb, 0));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float *out = a.partials + (size_t)blockIdx.x * (MLP_N_PARAMS + 1);
    if (ok) {
        // accumulator row tid (TMEM lane tid): weight rows, and the bias rows
        const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
        float v[16];
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 16) {
            tmem_ld16(lane + c0, v);
            for (int i = 0; i < 16; ++i) {
                if (tid < 12) out[OFF_W1 + tid * 64 + c0 + i] = v[i];
                else if (tid == 12) out[OFF_B1 + c0 + i] = v[i];
            }
            tmem_ld16(lane + 64u + c0, v);
            for (int i = 0; i < 16; ++i) {
                if (tid < 64) out[OFF_W2 + tid * 64 + c0 + i] = v[i];
                else if (tid == 64) out[OFF_B2 + c0 + i] = v[i];
            }
        }
        tmem_ld16(lane + 128u, v);
        for (int j = 0; j < 3; ++j) {
            if (tid < 64) out[OFF_W3 + tid * 3 + j] = v[j];
            else if (tid == 64) out[OFF_B3 + j] = v[j];
        }
    } else {
        if (tid == 0) atomicCAS(a.status, DEV_OK, DEV_ERR_TIMEOUT);
        mbar_wait(mb, 0);   // the MMAs still in flight, once more (bounded)
    }
    // loss of this block's samples, summed in a fixed tree order
    lsum[tid] = tid < cnt ? a.sample_loss[s0 + tid] : 0.f;
    __syncthreads();
    for (int w = WGRAD_CHUNK / 2; w > 0; w >>= 1) {
        if (tid < w) lsum[tid] += lsum[tid + w];
        __syncthreads();
    }
    if (tid == 0) out[MLP_N_PARAMS] = lsum[0];
    tc_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
}

__global__ void k_train_reduce(const float *partials, int blocks, int batch, float *grad_out,
                               float *loss_out, int adam, float *theta, float *m, float *v,
                               float lr, float beta1, float beta2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > MLP_N_PARAMS) return;
    float g = 0.f;
    for (int b = 0; b < blocks; ++b) g += partials[(size_t)b * (MLP_N_PARAMS + 1) + p];
    if (p == MLP_N_PARAMS) {
        if (loss_out) loss_out[0] = g / (3.f * (float)batch);
        return;
    }
    if (grad_out) grad_out[p] = g;
    if (!adam) return;
    const float mm = beta1 * m[p] + (1.f - beta1) * g;
    const float vv = beta2 * v[p] + (1.f - beta2) * g * g;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// the reduce of one Adam step with its step number read from device memory
__global__ void k_train_reduce_dev(const float *partials, int blocks, int batch, float *loss_hist,
                                   float *theta, float *m, float *v, float lr, float beta1,
                                   float beta2, float eps, const float *c12,
                                   const long long *step_dev) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > MLP_N_PARAMS) return;
    const long long t = *step_dev;
    float g = 0.f;
    for (int b = 0; b < blocks; ++b) g += partials[(size_t)b * (MLP_N_PARAMS + 1) + p];
    if (p == MLP_N_PARAMS) {
        loss_hist[t] = g / (3.f * (float)batch);
        return;
    }
    const float mm = beta1 * m[p] + (1.f - beta1) * g;
    const float vv = beta2 * v[p] + (1.f - beta2) * g * g;
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm * c12[2 * t]) / (sqrtf(vv * c12[2 * t + 1]) + eps);
}

// after every block of the reduce has read it
__global__ void k_step_advance(long long *step_dev) { *step_dev += 1; }

__global__ void k_loss_sum(const float *sample_loss, int n, double *acc) {
    __shared__ double part[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += sample_loss[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) acc[0] += part[0];
}

}  // namespace

void launch_depth(const uint64_t *mask, const int *row_ptr, const int *col, int n, uint8_t *depth,
                  cudaStream_t s) {
    if (n <= 0) return;
    const int grid = std::min((n + 255) / 256, 152 * 8);
    k_depth_init<<<grid, 256, 0, s>>>(mask, n, depth);
    note_launch();
    for (int L = 1; L < MLP_DEPTH_CAP; ++L) {
        k_depth_level<<<grid, 256, 0, s>>>(row_ptr, col, n, depth, L);
        note_launch();
    }
    CK(cudaGetLastError());
}

void launch_features(const FeatArgs &a, cudaStream_t s) {
    if (a.np <= 0) return;
    k_features<<<std::min((a.np + 255) / 256, 152 * 16), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

void launch_mlp_pack(const float *theta, uint32_t *packed, cudaStream_t s) {
    k_mlp_pack<<<1, 256, 0, s>>>(theta, packed);
    note_launch();
    CK(cudaGetLastError());
}

// Launch shape of the inference kernel on each device: the padding (dynamic
// shared bytes) that caps its CTAs per SM, the CTAs per SM and the SM count.
struct InferShape { int pad = 0, per_sm = 4, sms = 0; };
constexpr int kMaxDevices = 64;
InferShape g_infer[kMaxDevices];

void mlp_kernels_setup(int device) {
    if (device < 0 || device >= kMaxDevices) throw std::invalid_argument("device ordinal out of range");
    InferShape &g = g_infer[device];
    // At most 4 inference CTAs per SM: 4 x 128 tensor-memory columns fill an
    // SM's 512, and a fifth CTA would wait in tcgen05.alloc for a resident
    // one to finish.  Unused dynamic shared memory that makes a CTA take more
    // than a fifth of the SM's shared memory keeps the fifth off.
    int smem_sm = 0, reserved = 0;
    CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
    CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, k_mlp_infer<0>));
    const int need = smem_sm / 5 + 1 - (int)fa.sharedSizeBytes - reserved;
    const int pad = need > 0 ? (need + 15) & ~15 : 0;
    auto infer_attr = [&](const void *k) {
        CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, pad));
    };
    infer_attr((const void *)k_mlp_infer<0>);
    infer_attr((const void *)k_mlp_infer<1>);
    infer_attr((const void *)k_mlp_infer<2>);
    int occ = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_infer<0>, INFER_THREADS, pad));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    g.pad = pad;
    g.per_sm = std::max(1, std::min(occ, 4));
    g.sms = sms;
    CK(cudaFuncSetAttribute(k_train_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM));
    CK(cudaFuncSetAttribute(k_train_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, TF_SMEM));
}

void launch_mlp_infer(const uint32_t *packed, const float4 *feat, int n, int mode, float4 *lam0,
                      float *y3, int grid_limit, int *status, cudaStream_t s) {
    if (n <= 0) return;
    int device = -1;
    CK(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices || g_infer[device].sms == 0)
        throw std::logic_error("the network's kernels are not set up on this device");
    const InferShape &g = g_infer[device];   // set by mlp_kernels_setup
    const int kPad = g.pad;
    const int tiles = (n + 127) / 128;
    const int grid = std::min(tiles, grid_limit > 0 ? grid_limit : g.sms * g.per_sm);
    if (mode == 0) k_mlp_infer<0><<<grid, INFER_THREADS, kPad, s>>>(packed, feat, n, lam0, y3, status);
    else if (mode == 1) k_mlp_infer<1><<<grid, INFER_THREADS, kPad, s>>>(packed, feat, n, lam0, y3, status);
    else k_mlp_infer<2><<<grid, INFER_THREADS, kPad, s>>>(packed, feat, n, lam0, y3, status);
    note_launch();
    CK(cudaGetLastError());
}

void launch_log_append(const float4 *feat, const float4 *lam, const int *pos, int np,
                       float *log_feat, float *log_targ, long long base, long long cap,
                       cudaStream_t s) {
    if (np <= 0) return;
    k_log_append<<<std::min((np + 255) / 256, 152 * 16), 256, 0, s>>>(feat, lam, pos, np, log_feat,
                                                                        log_targ, base, cap);
    note_launch();
    CK(cudaGetLastError());
}

void launch_train_fwd(const TrainArgs &a, cudaStream_t s) {
    k_train_fwd<<<(a.batch + TRAIN_TILE - 1) / TRAIN_TILE, TRAIN_TILE, TF_SMEM, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

int train_wgrad_blocks(int batch) { return (batch + WGRAD_CHUNK - 1) / WGRAD_CHUNK; }

void launch_train_wgrad(const TrainArgs &a, cudaStream_t s) {
    k_train_wgrad<<<train_wgrad_blocks(a.batch), WGRAD_CHUNK, WG_SMEM, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

void launch_train_reduce(const float *partials, int blocks, int batch, float *grad_out,
                         float *loss_out, int adam, float *theta, float *m, float *v, float lr,
                         float beta1, float beta2, float eps, float c1, float c2, cudaStream_t s) {
    k_train_reduce<<<(MLP_N_PARAMS + 1 + 255) / 256, 256, 0, s>>>(
        partials, blocks, batch, grad_out, loss_out, adam, theta, m, v, lr, beta1, beta2, eps, c1, c2);
    note_launch();
    CK(cudaGetLastError());
}

void launch_train_reduce_dev(const float *partials, int blocks, int batch, float *loss_hist,
                             float *theta, float *m, float *v, float lr, float beta1, float beta2,
                             float eps, const float *c12, long long *step_dev, cudaStream_t s) {
    k_train_reduce_dev<<<(MLP_N_PARAMS + 1 + 255) / 256, 256, 0, s>>>(
        partials, blocks, batch, loss_hist, theta, m, v, lr, beta1, beta2, eps, c12, step_dev);
    note_launch();
    k_step_advance<<<1, 1, 0, s>>>(step_dev);
    note_launch();
    CK(cudaGetLastError());
}

void launch_loss_sum(const float *sample_loss, int n, double *acc, cudaStream_t s) {
    k_loss_sum<<<1, 256, 0, s>>>(sample_loss, n, acc);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
