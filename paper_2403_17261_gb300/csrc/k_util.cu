// k_util.cu -- scan, stable radix sort, fills and histograms used by the step.
#include "common.cuh"

#include <atomic>

namespace ovl {

namespace {
std::atomic<long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 2;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across the block (blockDim a
// multiple of 32); returns the block total through *total
__device__ int block_excl_scan(int v, int *total) {
    __shared__ int warp_sums[32];
    __shared__ int block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? warp_sums[lane] : 0;
        int wi = warp_incl_scan(w);
        warp_sums[lane] = wi - w;
        if (lane == 31) block_total = wi;
    }
    __syncthreads();
    int res = inc - v + warp_sums[warp];
    *total = block_total;
    __syncthreads();
    return res;
}

__global__ void k_tile_reduce(const int *in, int n, int *bsum) {
    int base = blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int i = base + threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    // block reduction
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = v;
    }
}

// single block: exclusive scan of nb block sums in place; total to *total_out
__global__ void k_scan_bsums(int *bsum, int nb, int *total_out) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int ex = block_excl_scan(v, &tot);
        if (i < nb) bsum[i] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_tile_scan(const int *in, int n, const int *bsum, int *out) {
    int base = blockIdx.x * SCAN_TILE;
    int vals[SCAN_ITEMS];
    int s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int i = base + threadIdx.x * SCAN_ITEMS + k;
        vals[k] = i < n ? in[i] : 0;
        s += vals[k];
    }
    int tot;
    int ex = block_excl_scan(s, &tot) + bsum[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int i = base + threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = ex;
        ex += vals[k];
    }
}

}  // namespace

void scan_i32(const int *in, int *out, int n, DBuf<int> &tmp, cudaStream_t s) {
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    tmp.ensure((size_t)nb + 1);
    k_tile_reduce<<<nb, SCAN_THREADS, 0, s>>>(in, n, tmp.p);
    note_launch();
    k_scan_bsums<<<1, SCAN_THREADS, 0, s>>>(tmp.p, nb, out + n);
    note_launch();
    k_tile_scan<<<nb, SCAN_THREADS, 0, s>>>(in, n, tmp.p, out);
    note_launch();
    CK(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_rs_hist(const uint32_t *keys, int n, int shift, int nblocks, int *hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint32_t *keys, const uint32_t *vals, int n, int shift,
                             int nblocks, const int *offs, uint32_t *keys_out, uint32_t *vals_out) {
    __shared__ int running[256];
    __shared__ int wcnt[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = 0;
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int i = base + r * RS_THREADS + tid;
        bool valid = i < n;
        uint32_t k = valid ? keys[i] : 0u;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & lt);
        if (valid && lrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        int pos = 0;
        if (valid) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
            pos = offs[d * nblocks + blockIdx.x] + running[d] + pre + lrank;
        }
        __syncthreads();
        {
            int add = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                add += wcnt[w][tid];
                wcnt[w][tid] = 0;
            }
            running[tid] += add;
        }
        if (valid) {
            keys_out[pos] = k;
            vals_out[pos] = vals[i];
        }
        __syncthreads();
    }
}

}  // namespace

void radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int n,
                    int nbits, DBuf<int> &hist, DBuf<int> &tmp, cudaStream_t s,
                    bool *result_in_alt) {
    *result_in_alt = false;
    if (n <= 1 || nbits <= 0) return;
    int nblocks = (n + RS_TILE - 1) / RS_TILE;
    hist.ensure((size_t)256 * nblocks + 1);
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_rs_hist<<<nblocks, RS_THREADS, 0, s>>>(ki, n, shift, nblocks, hist.p);
        note_launch();
        scan_i32(hist.p, hist.p, 256 * nblocks, tmp, s);
        k_rs_scatter<<<nblocks, RS_THREADS, 0, s>>>(ki, vi, n, shift, nblocks, hist.p, ko, vo);
        note_launch();
        CK(cudaGetLastError());
        uint32_t *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
        *result_in_alt = !*result_in_alt;
    }
}

namespace {
__global__ void k_fill_i32(int *p, int v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_fill_u8(uint8_t *p, uint8_t v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void k_iota(uint32_t *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = (uint32_t)i;
}
// bins privatised in shared memory (nbins <= 12288), one global add per bin and block
__global__ void k_hist(const int *key, int n, int *counts, int nbins) {
    extern __shared__ int h[];
    for (int j = threadIdx.x; j < nbins; j += blockDim.x) h[j] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&h[key[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < nbins; j += blockDim.x)
        if (h[j]) atomicAdd(&counts[j], h[j]);
}
__global__ void k_hist_global(const int *key, int n, int *counts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&counts[key[i]], 1);
}
int grid_for(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}
}  // namespace

void fill_i32(int *p, int v, size_t n, cudaStream_t s) {
    if (!n) return;
    k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    note_launch();
    CK(cudaGetLastError());
}
void fill_u8(uint8_t *p, uint8_t v, size_t n, cudaStream_t s) {
    if (!n) return;
    k_fill_u8<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    note_launch();
    CK(cudaGetLastError());
}
void iota_u32(uint32_t *p, int n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota<<<grid_for((size_t)n, 256), 256, 0, s>>>(p, n);
    note_launch();
    CK(cudaGetLastError());
}
void histogram_i32(const int *key, int n, int *counts, int nbins, cudaStream_t s) {
    if (!n) return;
    if (nbins <= 12288) {
        int g = grid_for((size_t)n, 256);
        if (g > 304) g = 304;
        k_hist<<<g, 256, (size_t)nbins * sizeof(int), s>>>(key, n, counts, nbins);
    } else {
        k_hist_global<<<grid_for((size_t)n, 256), 256, 0, s>>>(key, n, counts);
    }
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
