// common.cuh -- internal declarations shared by the libovl translation units.
//
// Device data layout (HBM):
//  * body state, 64 B per body (four float4, one 64-byte segment):
//      [0] px py pz radius   [1] qw qx qy qz   [2] vx vy vz inv_mass   [3] wx wy wz inv_inertia
//    The static lanes (radius, inverse mass, inverse inertia) ride in the
//    padding so one 64-byte gather brings a body's whole record.
//  * per-entry copies (one per (body, worker), Section 4's per-worker body
//    states) use the same 64-byte layout.
//  * contacts (canonical (a,b) order): int2 ab, float4 (n, phi), float4 (t1, 0).
//  * PGS rows of one worker, in colour order: four 16-byte records per
//    constraint plus a float4 of impulses (see k_solve.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ovl.h"

#define OVL_MAX_COLOURS 128
#define OVL_MAX_NEIGH 32   // sphere neighbours with larger index kept in registers per body; bodies
                           // whose neighbour capacity is larger continue in their global range

// device status codes (first error wins)
#define DEV_OK 0
#define DEV_ERR_CAPACITY 1
#define DEV_ERR_NONFINITE 2
#define DEV_ERR_MEMBERSHIP 3
#define DEV_ERR_COLOURS 4
#define DEV_ERR_TIMEOUT 5
#define DEV_ERR_SLOTS 6        // a worker of 2^24 or more bodies (beyond the slot codes)

namespace ovl {

struct CudaError {
    cudaError_t err;
    const char *what;
};

#define CK(x)                                                   \
    do {                                                        \
        cudaError_t e__ = (x);                                  \
        if (e__ != cudaSuccess) throw ::ovl::CudaError{e__, #x}; \
    } while (0)

// growable device buffer (contents are not preserved on growth)
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t cap = 0;
    // grows to twice the request: per-step sizes (pairs, entries) keep
    // rising while a pile settles, and every reallocation frees and maps
    // device memory (cudaFree waits for the device)
    void ensure(size_t n) {
        if (n <= cap && p) return;
        if (p) CK(cudaFree(p));
        size_t c = n < 16 ? 16 : 2 * n;
        CK(cudaMalloc(&p, c * sizeof(T)));
        cap = c;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// pinned host buffer
template <class T>
struct HBuf {
    T *p = nullptr;
    size_t cap = 0;
    void ensure(size_t n) {
        if (n <= cap && p) return;
        if (p) CK(cudaFreeHost(p));
        size_t c = n < 16 ? 16 : 2 * n;
        CK(cudaMallocHost(&p, c * sizeof(T)));
        cap = c;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

// kernel launches issued by this library (counted by every launcher)
void note_launch();
void note_launches(long long k);   // k kernels of a graph replay
long long launch_count();

// ---------------------------------------------------------------------------
// utility kernels (k_util.cu)
// ---------------------------------------------------------------------------
// exclusive scan of n int32 values; out has n+1 entries (out[n] = total)
void scan_i32(const int *in, int *out, int n, DBuf<int> &tmp, cudaStream_t s);
// stable LSD radix sort of (key, val) pairs by the low nbits of key
void radix_sort_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, int n,
                    int nbits, DBuf<int> &hist, DBuf<int> &tmp, cudaStream_t s,
                    bool *result_in_alt);
void fill_i32(int *p, int v, size_t n, cudaStream_t s);
void fill_u8(uint8_t *p, uint8_t v, size_t n, cudaStream_t s);
void iota_u32(uint32_t *p, int n, cudaStream_t s);
// counts[key[i]]++ for i < n
void histogram_i32(const int *key, int n, int *counts, int nbins, cudaStream_t s);

// ---------------------------------------------------------------------------
// host-side algorithms (host_alg.cpp): Algorithms 2, 3, 6, 7
// ---------------------------------------------------------------------------
struct HostScene {
    int n = 0, ns = 0, n_parts = 0;
    std::vector<float> inv_mass;
    std::vector<int> sob, part_base, scene_gamma, n_sets;
    std::vector<int> body_base;  // [ns+1] first body of every scene
    std::vector<int> jab;  // 2 per joint
};

// breadth-first workspaces of the load balance, one per host thread, kept
// across steps (epoch-stamped, so never cleared)
struct BallWorkspace {
    std::vector<int> seen, out;
    int epoch = 0;
};

void host_assign_overlap(const HostScene &sc, std::vector<uint64_t> &mask);
// contacts ab: pairs of dynamic bodies in canonical order; graph CSR of G^t;
// mask [n] updated in place; loads [n_parts]: |P_w| of every worker for
// these masks; scenes spread over up to `threads` threads (ws.size()).
// ball_start [n+1] / ball_vtx (both NULL, or both set): the gamma-ball of
// body v found beforehand at ball_vtx[ball_start[v] .. ball_start[v+1]);
// an empty range means the pass searches that ball itself.
void host_load_balance(const HostScene &sc, uint64_t *mask, const int *loads, const int *deg, int64_t nc,
                       const int2 *ab, const int *row_ptr, const int *col, bool do_activate,
                       bool do_deactivate, std::vector<BallWorkspace> &ws, const int *ball_start = nullptr,
                       const int *ball_vtx = nullptr);

}  // namespace ovl
