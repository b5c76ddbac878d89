// k_geo_static.cu -- geodesic distances D(o,i) (Eq 16, Algorithm 5) for one
// scene, with all scratch in a statically sized __device__ array so that the
// call allocates no device memory.
//
// The search is the same level-synchronous multi-source BFS as the geodesic
// phase of a step: a queue item is (body, worker), level 0 holds every body
// whose mask is the single worker i as (b, i), and a bit per (worker, body)
// marks the pairs already reached, so the level at which (o, i) is first
// reached is the graph distance from o to the nearest body of worker i alone.
// Differences: one scene only, scratch from the static array below instead
// of the context's buffers, and every index read from a caller's array is
// range-checked before it is used.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "ovl.h"

namespace {

constexpr long long kMaxPairs = OVL_GEO_STATIC_MAX_PAIRS;
constexpr int kMaxBeta = OVL_GEO_STATIC_MAX_BETA;
static_assert(kMaxPairs % 32 == 0, "bitmap words");
static_assert(kMaxPairs <= (1ll << 26), "queue items hold a body index in 26 bits");
static_assert(kMaxBeta <= 254, "D is a byte and 255 means not reached");

struct GeoScratch {
    uint32_t visited[kMaxPairs / 32];  // bit w * n + b: (body b, worker w) reached
    uint32_t queue[kMaxPairs];         // (b << 6) | w, each pair enqueued at most once
    int qctl[kMaxBeta + 4];            // [0] tail, [1 + L] first queue index of level L
};

// 16.5 MiB of device memory, reserved when the module is loaded.
static __device__ __align__(256) GeoScratch g_geo_scratch;

struct GeoIn {
    int n, nw, n_adj, ne;
    uint64_t wmask;  // bits of workers 0 .. nw-1
    const int *row_ptr, *col, *entry_ptr;
    const uint64_t *mask;
    uint8_t *D;
};

__device__ __forceinline__ bool claim(uint32_t *visited, long long bit) {
    const uint32_t m = 1u << (bit & 31);
    return !(atomicOr(&visited[bit >> 5], m) & m);
}

__device__ __forceinline__ void enqueue(int *tail, uint32_t *queue, uint32_t item) {
    const unsigned active = __activemask();
    const int leader = __ffs(active) - 1, lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(tail, __popc(active));
    base = __shfl_sync(active, base, leader);
    queue[base + __popc(active & ((1u << lane) - 1u))] = item;
}

// Zeroes the bitmap words and level counters this call uses; D := 255.
__global__ void k_gs_clear(GeoScratch *s, long long words, int nctl, uint8_t *D, int ne) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words; i += stride)
        s->visited[i] = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ne; i += stride)
        D[i] = 255;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < nctl; i += blockDim.x) s->qctl[i] = 0;
}

__global__ void k_gs_sources(GeoScratch *s, GeoIn in) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < in.n; b += gridDim.x * blockDim.x) {
        const uint64_t m = in.mask[b] & in.wmask;
        if (__popcll(m) != 1) continue;
        const int w = __ffsll((long long)m) - 1;
        claim(s->visited, (long long)w * in.n + b);
        enqueue(&s->qctl[0], s->queue, ((uint32_t)b << 6) | (uint32_t)w);
    }
}

__global__ void k_gs_mark(GeoScratch *s, int level) { s->qctl[1 + level] = s->qctl[0]; }

// Expands the items of level-1 into level `level`: one warp per item.
__global__ void k_gs_level(GeoScratch *s, GeoIn in, int level, int last) {
    const int start = s->qctl[level], end = s->qctl[1 + level];
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int it = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) + start; it < end; it += warps) {
        const uint32_t item = s->queue[it];
        const int u = (int)(item >> 6), w = (int)(item & 63u);
        const int k0 = max(in.row_ptr[u], 0), k1 = min(in.row_ptr[u + 1], in.n_adj);
        for (int k = k0 + lane; k < k1; k += 32) {
            const int v = in.col[k];
            if (v < 0 || v >= in.n) continue;
            if (!claim(s->visited, (long long)w * in.n + v)) continue;
            const uint64_t mv = in.mask[v] & in.wmask;
            if (__popcll(mv) >= 2 && (mv >> w & 1ull)) {
                const int e = in.entry_ptr[v] + __popcll(mv & ((1ull << w) - 1ull));
                if (e >= 0 && e < in.ne) in.D[e] = (uint8_t)level;
            }
            if (!last) enqueue(&s->qctl[0], s->queue, ((uint32_t)v << 6) | (uint32_t)w);
        }
    }
}

int report(char *err, int cap, int code, const char *msg) {
    if (err && cap > 0) snprintf(err, (size_t)cap, "%s", msg);
    return code;
}

// The device address of the scratch array in the current device's context.
// It is looked up on every call, not cached per device number: a device reset
// (cudaDeviceReset) or a released and re-created primary context reloads the
// module, and the array may then sit at another address.  After the module is
// loaded the lookup is a table read.
int scratch_of_current_device(GeoScratch **out, char *err, int cap) {
    GeoScratch *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_geo_scratch);
    if (e != cudaSuccess || !p) {
        char msg[160];
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the geodesic scratch failed: %s",
                 cudaGetErrorString(e));
        return report(err, cap, OVL_ERR_CUDA, msg);
    }
    *out = p;
    return OVL_OK;
}

}  // namespace

extern "C" ovl_status ovl_geodesics_static(int32_t n_bodies, int32_t n_workers, int32_t beta,
                                           const int32_t *row_ptr, const int32_t *col,
                                           int32_t n_adj, const uint64_t *mask,
                                           const int32_t *entry_ptr, int32_t n_entries,
                                           uint8_t *D, void *cuda_stream, char *err,
                                           int32_t err_cap) {
    if (err && err_cap > 0) err[0] = '\0';
    if (n_bodies < 0 || n_adj < 0 || n_entries < 0)
        return report(err, err_cap, OVL_ERR_ARG, "negative size");
    if (n_workers < 1 || n_workers > 64)
        return report(err, err_cap, OVL_ERR_ARG, "n_workers must be in [1, 64]");
    if (beta < 0) return report(err, err_cap, OVL_ERR_ARG, "beta must be >= 0");
    if (beta > kMaxBeta) {
        char msg[128];
        snprintf(msg, sizeof msg, "beta = %d exceeds OVL_GEO_STATIC_MAX_BETA = %d", beta, kMaxBeta);
        return report(err, err_cap, OVL_ERR_CAPACITY, msg);
    }
    const long long pairs = (long long)n_bodies * n_workers;
    if (pairs > kMaxPairs) {
        char msg[160];
        snprintf(msg, sizeof msg,
                 "n_bodies * n_workers = %lld exceeds OVL_GEO_STATIC_MAX_PAIRS = %lld", pairs,
                 kMaxPairs);
        return report(err, err_cap, OVL_ERR_CAPACITY, msg);
    }
    if ((n_bodies > 0 && (!row_ptr || !mask || !entry_ptr)) || (n_adj > 0 && !col) ||
        (n_entries > 0 && !D))
        return report(err, err_cap, OVL_ERR_ARG, "null array with a nonzero size");
    if (n_bodies == 0 && n_entries == 0) return OVL_OK;

    GeoScratch *s = nullptr;
    int rc = scratch_of_current_device(&s, err, err_cap);
    if (rc != OVL_OK) return rc;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    GeoIn in{};
    in.n = n_bodies; in.nw = n_workers; in.n_adj = n_adj; in.ne = n_entries;
    in.wmask = n_workers >= 64 ? ~0ull : ((1ull << n_workers) - 1ull);
    in.row_ptr = row_ptr; in.col = col; in.entry_ptr = entry_ptr; in.mask = mask; in.D = D;

    const long long words = (pairs + 31) / 32;
    const long long widest = words > n_entries ? words : n_entries;
    const int clear_blocks = (int)(widest / 256 + 1 < 152 * 8 ? widest / 256 + 1 : 152 * 8);
    k_gs_clear<<<clear_blocks, 256, 0, st>>>(s, words, beta + 3, D, n_entries);
    if (n_bodies > 0) {
        const int src_blocks = (n_bodies + 255) / 256 < 152 * 8 ? (n_bodies + 255) / 256 : 152 * 8;
        k_gs_sources<<<src_blocks, 256, 0, st>>>(s, in);
        k_gs_mark<<<1, 1, 0, st>>>(s, 1);
        for (int L = 1; L <= beta; ++L) {
            k_gs_level<<<152 * 8, 256, 0, st>>>(s, in, L, L == beta);
            k_gs_mark<<<1, 1, 0, st>>>(s, L + 1);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(err, err_cap, OVL_ERR_CUDA, cudaGetErrorString(e));
    return OVL_OK;
}
