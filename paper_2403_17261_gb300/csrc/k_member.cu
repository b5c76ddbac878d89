// k_member.cu -- who solves what (Section 4, Eq 9-10): membership entries
// (body, worker), every worker's body list and local slots, the
// (worker, constraint) pairs with their warm-start impulses, the per-worker
// colouring that orders the Gauss-Seidel sweep, and the colour-ordered row
// records the solver streams.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"
#include "geom.cuh"

namespace cg = cooperative_groups;

namespace ovl {

namespace {

__device__ __forceinline__ uint64_t cons_mask(int i, int nc, int n, const int2 *c_ab, const int2 *jab,
                                              const float *im, const uint64_t *mask) {
    int2 e = i < nc ? c_ab[i] : jab[i - nc];
    bool da = e.x >= 0 && e.x < n && im[e.x] > 0.0f;
    bool db = e.y >= 0 && e.y < n && im[e.y] > 0.0f;
    if (!da && !db) return 0;
    uint64_t m = ~0ull;
    if (da) m &= mask[e.x];
    if (db) m &= mask[e.y];
    return m;
}

__device__ __forceinline__ int cons_scene(int i, int nc, const int2 *c_ab, const int *sob,
                                          const int *joint_scene) {
    return i < nc ? sob[c_ab[i].x] : joint_scene[i - nc];
}

__global__ void k_entry_count(MemberArgs a) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.n; b += gridDim.x * blockDim.x) {
        uint64_t m = a.mask[b];
        int ns = a.n_sets[a.sob[b]];
        uint64_t allowed = ns >= 64 ? ~0ull : ((1ull << ns) - 1ull);
        bool dyn = a.im[b] > 0.0f;
        if ((dyn && m == 0) || (m & ~allowed) || (!dyn && m)) atomicCAS(a.status, DEV_OK, DEV_ERR_MEMBERSHIP);
        a.entry_count[b] = dyn ? __popcll(m & allowed) : 0;
    }
}

__global__ void k_entry_fill(MemberArgs a) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.n; b += gridDim.x * blockDim.x) {
        int e = a.entry_ptr[b];
        int cnt = a.entry_ptr[b + 1] - e;
        int ns = a.n_sets[a.sob[b]];
        uint64_t m = a.mask[b] & (ns >= 64 ? ~0ull : ((1ull << ns) - 1ull));
        int base = a.part_base[a.sob[b]];
        for (int k = 0; k < cnt; ++k) {
            int w = __ffsll((long long)m) - 1;
            m &= m - 1;
            a.entry_body[e + k] = b;
            a.entry_part[e + k] = base + w;
        }
    }
}

__global__ void k_entry_slot(MemberArgs a, int ne) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
        int e = a.part_list[k];
        a.entry_slot[e] = k - a.part_bstart[a.entry_part[e]];
    }
}

__global__ void k_cons_count(MemberArgs a) {
    int total = a.nc + a.nj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        a.cons_count[i] = __popcll(cons_mask(i, a.nc, a.n, a.c_ab, a.jab, a.im, a.mask));
}

__global__ void k_pair_fill(MemberArgs a) {
    int total = a.nc + a.nj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        uint64_t m = cons_mask(i, a.nc, a.n, a.c_ab, a.jab, a.im, a.mask);
        int q = a.cons_start[i];
        int base = a.part_base[cons_scene(i, a.nc, a.c_ab, a.sob, a.joint_scene)];
        while (m) {
            int w = __ffsll((long long)m) - 1;
            m &= m - 1;
            a.pair_cons[q] = i;
            a.pair_part[q] = base + w;
            ++q;
        }
    }
}

__global__ void k_pair_gather(MemberArgs a, const uint32_t *order, int np) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        int q = (int)order[k];
        a.ps_cons[k] = a.pair_cons[q];
        a.ps_part[k] = a.pair_part[q];
    }
}

__device__ __forceinline__ int body_slot(const MemberArgs &a, int x, int w) {
    if (x < 0 || x >= a.n || !(a.im[x] > 0.0f)) return -1;
    uint64_t m = a.mask[x];
    int e = a.entry_ptr[x] + __popcll(m & ((1ull << w) - 1ull));
    return a.entry_slot[e];
}

// One block per (worker, colour); warp w takes the w-th contiguous chunk of
// the colour's rows.  A row's owner is the CTA that holds its first dynamic
// body.  The warps count their rows per (owner rank, kind); a colour step
// lasts as long as its fullest CTA, so a CTA with more rows of a kind than
// the even share (total / C) passes half of the excess on: it keeps its own
// rows up to its new share, in order, and the rows beyond it go, in order, to
// the CTAs below the even share (after those CTAs' own rows), which reach
// their bodies in the owner's shared memory.  (Measured on the large pile:
// moving the whole excess saved less, the remote accesses cost more than the
// balance gained.)  Buckets
// are laid out rank by rank (contacts, then joints).  Rows of one colour are
// independent, so any assignment gives the same result.
constexpr int OWNER_THREADS = 256, OWNER_WARPS = OWNER_THREADS / 32;

__global__ void __launch_bounds__(OWNER_THREADS)
k_row_owner(int P, const int *part_bstart, const int *part_ncol, const int *solve_C,
            const int *off_in, const int *pair_of_row, const int2 *p_slot, uint8_t *owner_of_row,
            int *pair_of_row_out, int *off_out) {
    constexpr int NK = 2 * OWNER_RANKS;
    __shared__ int cnt[OWNER_WARPS][NK];    // a warp's rows per (owner, kind), then its first index in the group
    __shared__ int total[NK], share[NK], start[NK], exc0[NK], def0[NK];
    const int p = blockIdx.x, c = blockIdx.y;
    if (p >= P) return;
    const int ncol = part_ncol[p];
    const int *off = off_in + (size_t)p * (2 * OVL_MAX_COLOURS + 1);
    int *o2 = off_out + (size_t)p * OWNER_NB;
    const int end = off[2 * ncol];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (c >= ncol) {
        if (tid < NK) o2[c * NK + tid] = end;
        if (c == OVL_MAX_COLOURS - 1 && tid == 0) o2[OWNER_NB - 1] = end;
        return;
    }
    const int nb = part_bstart[p + 1] - part_bstart[p];
    const int C = max(1, min(solve_C[p], OWNER_RANKS));
    const int per = max(1, (nb + C - 1) / C);
    const int s0 = off[2 * c], s1 = off[2 * c + 1], s2 = off[2 * c + 2];
    const int chunk = (s2 - s0 + OWNER_WARPS - 1) / OWNER_WARPS;
    const int w0 = min(s2, s0 + warp * chunk), w1 = min(s2, w0 + chunk);
    if (lane < NK) cnt[warp][lane] = 0;
    __syncwarp();
    const unsigned full = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    // bucket of a row: 2 owner + kind (0 contact, 1 joint)
    for (int b = w0; b < w1; b += 32) {
        const int r = b + lane;
        int key = -1;
        if (r < w1) {
            const int2 sl = p_slot[pair_of_row[r]];
            const int sa = sl.x >= 0 ? sl.x : max(sl.y, 0);
            key = 2 * min(sa / per, C - 1) + (r >= s1 ? 1 : 0);
            owner_of_row[r] = (uint8_t)key;
        }
        const unsigned peers = __match_any_sync(full, key);
        if (key >= 0 && (peers & lt) == 0) cnt[warp][key] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NK; ++k) {
            int t = 0;
            for (int w = 0; w < OWNER_WARPS; ++w) {   // counts -> each warp's first index in its group
                const int x = cnt[w][k];
                cnt[w][k] = t;
                t += x;
            }
            total[k] = t;
        }
        for (int kind = 0; kind < 2; ++kind) {
            int all = 0;
            for (int r = 0; r < OWNER_RANKS; ++r) all += total[2 * r + kind];
            // a CTA above the even share passes on half of its excess; the
            // CTAs below it take those rows in rank order
            int moved = 0;
            for (int r = 0; r < OWNER_RANKS; ++r) {
                const int k = 2 * r + kind;
                const int even = r < C ? all / C + (r < all % C ? 1 : 0) : 0;
                share[k] = total[k] > even ? total[k] - (total[k] - even) / 2 : even;
                moved += total[k] - min(total[k], share[k]);
            }
            int e = 0, d = 0;
            for (int r = 0; r < OWNER_RANKS; ++r) {
                const int k = 2 * r + kind;
                if (share[k] > total[k]) {
                    const int take = min(share[k] - total[k], moved);
                    share[k] = total[k] + take;
                    moved -= take;
                }
                exc0[k] = e;
                def0[k] = d;
                e += max(0, total[k] - share[k]);
                d += max(0, share[k] - total[k]);
            }
        }
        int pos = s0;
        for (int k = 0; k < NK; ++k) {
            start[k] = pos;
            o2[c * NK + k] = pos;
            pos += share[k];
        }
        if (c == OVL_MAX_COLOURS - 1) o2[OWNER_NB - 1] = end;
    }
    __syncthreads();
    for (int b = w0; b < w1; b += 32) {
        const int r = b + lane;
        const int key = r < w1 ? (int)owner_of_row[r] : -1;
        const unsigned peers = __match_any_sync(full, key);
        if (key >= 0) {
            const int idx = cnt[warp][key] + __popc(peers & lt);   // index in its (owner, kind) group
            int dst;
            if (idx < share[key]) {
                dst = start[key] + idx;
            } else {
                // the e-th row beyond its owner's share (over owners in rank
                // order) fills the e-th free place of the same kind
                const int kind = key & 1;
                const int e = exc0[key] + (idx - share[key]);
                int k = kind;
                while (k + 2 < NK && def0[k + 2] <= e) k += 2;
                dst = start[k] + total[k] + (e - def0[k]);
            }
            pair_of_row_out[dst] = pair_of_row[r];
        }
        __syncwarp();
        if (key >= 0 && (peers & lt) == 0) cnt[warp][key] += __popc(peers);
        __syncwarp();
    }
}

__global__ void k_worker_cost_keys(const int *part_pstart, int P, uint32_t *keys, uint32_t *vals) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const uint32_t cost = (uint32_t)min(part_pstart[p + 1] - part_pstart[p], (1 << 24) - 1);
        keys[p] = ((1u << 24) - 1u) - cost;
        vals[p] = (uint32_t)p;
    }
}

// manifold index of contact i (0 without boxes)
__device__ __forceinline__ int contact_point(const MemberArgs &a, int i) {
    return a.c_p ? __float_as_int(a.c_p[i].w) : 0;
}

__global__ void k_pair_setup(MemberArgs a, WarmArgs ws, int np) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        int i = a.ps_cons[k], p = a.ps_part[k];
        int scene = cons_scene(i, a.nc, a.c_ab, a.sob, a.joint_scene);
        int w = p - a.part_base[scene];
        int2 e;
        uint64_t key;
        if (i < a.nc) {
            e = a.c_ab[i];
            // a << 32 | b << 2 | k: key order is the canonical contact order
            key = ((uint64_t)(uint32_t)e.x << 32) | ((uint64_t)(uint32_t)e.y << 2) | (uint64_t)contact_point(a, i);
        } else {
            e = a.jab[i - a.nc];
            key = (1ull << 62) | (uint64_t)(i - a.nc);
        }
        a.p_key[k] = key;
        a.p_slot[k] = make_int2(body_slot(a, e.x, w), body_slot(a, e.y, w));
        // warm start: the previous step's impulses of the same (worker, key)
        int lo = ws.ws_pstart[p], hi = ws.ws_pstart[p + 1];
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (ws.ws_key[mid] < key) lo = mid + 1; else hi = mid;
        }
        float4 l0 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lo < ws.ws_pstart[p + 1] && ws.ws_key[lo] == key) {
            float4 v = ws.ws_lam[lo];
            l0 = make_float4(v.x * ws.factor, v.y * ws.factor, v.z * ws.factor, 0.f);
        }
        a.p_lam0[k] = l0;
    }
}

// ---------------------------------------------------------------------------
// Colouring: Jones-Plassmann with first-fit colours.  A constraint takes its
// colour once every constraint of higher priority sharing one of its dynamic
// bodies is coloured; it takes the smallest colour none of them holds.  This
// assigns exactly the colours of a sequential greedy pass in descending
// priority (the constraints coloured before it are then exactly its
// higher-priority neighbours).  Priority = SplitMix64 finaliser of the key.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int COLOUR_THREADS = 1024;
constexpr int COLOUR_WARPS = COLOUR_THREADS / 32;
constexpr int NBUCKET = 2 * OVL_MAX_COLOURS;

__device__ __forceinline__ uint32_t mapa_u32(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// Per-slot colouring state of one worker: the maximum priority of the
// uncoloured constraints posted this round (array 0) and the mask of colours
// 0-63 taken (array 1).  Colours 64-127, which only bodies in about 64 or
// more constraints need, are tracked in global memory (hi_mask).
// C > 1: spread over the cluster's shared memory, CTA k holding the
// contiguous slots [k per, (k + 1) per).  The
// maximum is taken in two 32-bit stages (high words, then low words among the
// constraints whose high word won), which is the 64-bit maximum: 64-bit atomic
// max into another CTA's shared memory lost updates in a standalone test on
// this GPU, 32-bit ones did not.
template <int C>
struct ColourSlots {
    static constexpr bool two_stage = true;
    uint32_t b0, b1;   // shared-window offsets of this CTA's arrays (hi/lo words, used mask)
    int per;           // slots per CTA
    __device__ __forceinline__ uint32_t at(int arr, int s) const {
        uint32_t base = arr == 0 ? b0 : b1;
        uint32_t r = 0;
#pragma unroll
        for (int k = 1; k < C; ++k) r += s >= k * per ? 1u : 0u;
        return mapa_u32(base + 8u * ((uint32_t)s - r * (uint32_t)per), r);
    }
    // stage 1: high word (at offset +4 of the little-endian 64-bit slot)
    __device__ __forceinline__ void amax_hi(int s, unsigned long long v) const {
        asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(at(0, s) + 4u), "r"((uint32_t)(v >> 32)) : "memory");
    }
    __device__ __forceinline__ void amax_lo(int s, unsigned long long v) const {
        asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(at(0, s)), "r"((uint32_t)v) : "memory");
    }
    __device__ __forceinline__ uint32_t ld_hi(int s) const {
        uint32_t v;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(at(0, s) + 4u) : "memory");
        return v;
    }
    __device__ __forceinline__ unsigned long long ld(int arr, int s) const {
        unsigned long long v;
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(at(arr, s)) : "memory");
        return v;
    }
    __device__ __forceinline__ void st(int arr, int s, unsigned long long v) const {
        asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(at(arr, s)), "l"(v) : "memory");
    }
};

// One CTA: shared or global memory through plain pointers (volatile reads so
// that values written by other threads' atomics are seen after a barrier);
// one 64-bit atomic max per slot.
struct ColourPtrs {
    static constexpr bool two_stage = false;
    unsigned long long *p0, *p1;
    __device__ __forceinline__ unsigned long long *ptr(int arr, int s) const {
        return (arr == 0 ? p0 : p1) + s;
    }
    __device__ __forceinline__ void amax_hi(int s, unsigned long long v) const { atomicMax(ptr(0, s), v); }
    __device__ __forceinline__ void amax_lo(int, unsigned long long) const {}
    __device__ __forceinline__ uint32_t ld_hi(int s) const {
        return (uint32_t)(*reinterpret_cast<volatile unsigned long long *>(ptr(0, s)) >> 32);
    }
    __device__ __forceinline__ unsigned long long ld(int arr, int s) const {
        return *reinterpret_cast<volatile unsigned long long *>(ptr(arr, s));
    }
    __device__ __forceinline__ void st(int arr, int s, unsigned long long v) const { *ptr(arr, s) = v; }
};

template <int C>
__device__ __forceinline__ void csync() {
    if (C == 1) __syncthreads();
    else cg::this_cluster().sync();
}

// sum over the group's CTAs of one int per CTA held in shared variable *v
template <int C>
__device__ __forceinline__ int cluster_int_sum(int *v) {
    if (C == 1) return *v;
    cg::cluster_group cl = cg::this_cluster();
    int t = 0;
    for (int r = 0; r < C; ++r) t += *cl.map_shared_rank(v, r);
    return t;
}

// Colours one worker with a group of C CTAs.  CTA `rank` holds the slots
// [rank per, (rank + 1) per) and takes two contiguous shares of the worker's
// constraints (canonical order: contacts by their first body, then joints):
// the contacts whose first body falls in its slot range, so most of their
// slot accesses stay local, and an equal share of the joints.  The shares
// follow rank order, so the final sort is stable across CTAs.
// The CTA's static shared state, declared once in the kernel: both
// instantiations of colour_worker (cluster slots and the global-memory
// fallback) share it instead of each holding its own copy.
struct ColourShared {
    int n_next, ncol_sh, pub_left[2], pub_ncol;   // pub_left: by round parity
    int counts[NBUCKET + 1];
    int base_b[NBUCKET + 1];
    int running[NBUCKET];
    uint8_t wcnt[COLOUR_WARPS][NBUCKET];   // one warp's items per bucket (at most 32)
};

template <int C, class SL>
__device__ void colour_worker(const ColourArgs &a, const SL &S, ColourShared &sh, int p, int rank, int per) {
    int &n_next = sh.n_next, &ncol_sh = sh.ncol_sh, &pub_ncol = sh.pub_ncol;
    int *pub_left = sh.pub_left;
    int (&counts)[NBUCKET + 1] = sh.counts;
    int (&base_b)[NBUCKET + 1] = sh.base_b;
    int (&running)[NBUCKET] = sh.running;
    uint8_t (&wcnt)[COLOUR_WARPS][NBUCKET] = sh.wcnt;
    const int tid = threadIdx.x, T = blockDim.x;
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    const int q0 = a.part_pstart[p], nq = a.part_pstart[p + 1] - q0;
    const int s_lo = C == 1 ? 0 : min(nb, rank * per), s_hi = C == 1 ? nb : min(nb, (rank + 1) * per);
    // contacts [0, ncw) are sorted by (first body, second body), joints [ncw, nq) by index
    const uint64_t *key = a.p_key + q0;
    auto key_bound = [&](int lo, int hi, uint64_t x) {
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (key[mid] < x) lo = mid + 1; else hi = mid; }
        return lo;
    };
    const int ncw = key_bound(0, nq, 1ull << 62);
    auto first_contact = [&](int k) {   // first contact whose first body is in slot range k or later
        if (k <= 0) return 0;
        if (k * per >= nb) return ncw;
        const uint64_t body = (uint64_t)a.entry_body[a.part_list[b0 + k * per]];
        return key_bound(0, ncw, body << 32);
    };
    const int c0 = C == 1 ? 0 : first_contact(rank), c1 = C == 1 ? ncw : first_contact(rank + 1);
    const int jchunk = (nq - ncw + C - 1) / C;
    const int j0 = min(nq, ncw + rank * jchunk), j1 = min(nq, j0 + jchunk);
    const int nC = c1 - c0, m0 = nC + (j1 - j0);
    auto item = [&](int v) { return v < nC ? c0 + v : j0 + (v - nC); };
    // worklists of this CTA's uncoloured constraints: (index in worker,
    // slot a, slot b) and the priority, ping-pong, read contiguously; the
    // CTA's region follows the regions of the lower ranks
    const int wbase = c0 + (j0 - ncw);
    int4 *wl_cur = a.worklist + q0 + wbase, *wl_next = a.worklist2 + q0 + wbase;
    unsigned long long *pr_cur = a.wprio + q0 + wbase, *pr_next = a.wprio2 + q0 + wbase;
    // colours 64-127 of the worker's slots (global memory, read past L1: other
    // CTAs of the group write them)
    unsigned long long *hi = a.hi_mask + b0;
    for (int s = s_lo + tid; s < s_hi; s += T) { S.st(1, s, 0ull); __stcg(hi + s, 0ull); }
    for (int v = tid; v < m0; v += T) {
        const int k = item(v);
        int2 sl = a.p_slot[q0 + k];
        wl_cur[v] = make_int4(k, sl.x, sl.y, 0);
        pr_cur[v] = mix64(key[k]);
    }
    if (tid == 0) { n_next = 0; ncol_sh = 0; }
    int m = m0;
    int rounds = 0;
    // Every round: each CTA zeroes the maxima of the slots it holds, all
    // uncoloured constraints post their priority at their slots, and those
    // holding the maximum at both slots take their colour.
    while (rounds <= nq + 1) {
        for (int s = s_lo + tid; s < s_hi; s += T) S.st(0, s, 0ull);
        csync<C>();
        for (int i = tid; i < m; i += T) {
            const int4 w = wl_cur[i];
            const unsigned long long pr = pr_cur[i];
            if (w.y >= 0) S.amax_hi(w.y, pr);
            if (w.z >= 0) S.amax_hi(w.z, pr);
        }
        csync<C>();
        if (SL::two_stage) {
            for (int i = tid; i < m; i += T) {
                const int4 w = wl_cur[i];
                const unsigned long long pr = pr_cur[i];
                const uint32_t hi = (uint32_t)(pr >> 32);
                if (w.y >= 0 && S.ld_hi(w.y) == hi) S.amax_lo(w.y, pr);
                if (w.z >= 0 && S.ld_hi(w.z) == hi) S.amax_lo(w.z, pr);
            }
            csync<C>();
        }
        for (int i = tid; i < m; i += T) {
            const int4 w = wl_cur[i];
            const unsigned long long pr = pr_cur[i];
            bool ready = (w.y < 0 || S.ld(0, w.y) == pr) && (w.z < 0 || S.ld(0, w.z) == pr);
            if (!ready) {
                int o = atomicAdd(&n_next, 1);
                wl_next[o] = w;
                pr_next[o] = pr;
                continue;
            }
            // only this constraint touches its slots in this round
            unsigned long long u = 0ull;   // colours 0-63 taken at its slots
            if (w.y >= 0) u |= S.ld(1, w.y);
            if (w.z >= 0) u |= S.ld(1, w.z);
            int c;
            if (~u) {
                c = __ffsll((long long)~u) - 1;
                const unsigned long long bit = 1ull << c;
                if (w.y >= 0) S.st(1, w.y, S.ld(1, w.y) | bit);
                if (w.z >= 0) S.st(1, w.z, S.ld(1, w.z) | bit);
            } else {
                unsigned long long v = 0ull;   // colours 64-127
                if (w.y >= 0) v |= __ldcg(hi + w.y);
                if (w.z >= 0) v |= __ldcg(hi + w.z);
                if (~v) {
                    c = 64 + __ffsll((long long)~v) - 1;
                } else {
                    c = OVL_MAX_COLOURS - 1;
                    atomicCAS(a.status, DEV_OK, DEV_ERR_COLOURS);
                }
                const unsigned long long bit = 1ull << (c - 64);
                if (w.y >= 0) __stcg(hi + w.y, __ldcg(hi + w.y) | bit);
                if (w.z >= 0) __stcg(hi + w.z, __ldcg(hi + w.z) | bit);
            }
            a.p_colour[q0 + w.x] = c;
            atomicMax(&ncol_sh, c + 1);
        }
        __syncthreads();
        // the count of this round goes to pub_left[rounds & 1]: it is written
        // again two rounds later, after the barriers of the next round, which
        // every CTA passes only once it has summed this one
        if (tid == 0) pub_left[rounds & 1] = n_next;
        csync<C>();
        const int left = cluster_int_sum<C>(&pub_left[rounds & 1]);
        m = n_next;
        ++rounds;
        __syncthreads();
        if (tid == 0) n_next = 0;
        { int4 *t = wl_cur; wl_cur = wl_next; wl_next = t; }
        { unsigned long long *t = pr_cur; pr_cur = pr_next; pr_next = t; }
        if (left == 0) break;
    }
    if (rank == 0 && tid == 0 && rounds > nq + 1) atomicCAS(a.status, DEV_OK, DEV_ERR_TIMEOUT);
    // stable counting sort of the worker's constraints by (colour, kind):
    // contacts before joints inside a colour, canonical order kept; CTA r's
    // share goes after the shares of lower ranks in every bucket
    for (int j = tid; j <= NBUCKET; j += T) counts[j] = 0;
    for (int j = tid; j < NBUCKET; j += T) running[j] = 0;
    for (int j = tid; j < COLOUR_WARPS * NBUCKET; j += T) (&wcnt[0][0])[j] = 0;
    __syncthreads();
    for (int v = tid; v < m0; v += T) {
        const int k = item(v);
        int c = a.p_colour[q0 + k];
        int kind = (int)(key[k] >> 62) & 1;
        atomicAdd(&counts[2 * c + kind], 1);
    }
    if (tid == 0) pub_ncol = ncol_sh;
    csync<C>();
    // bucket base of this CTA: all earlier buckets of every CTA, plus this
    // bucket in lower-ranked CTAs
    for (int j = tid; j <= NBUCKET; j += T) {
        int before = 0, lower = 0;
        if (C == 1) {
            for (int jj = 0; jj < j; ++jj) before += counts[jj];
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int r = 0; r < C; ++r) {
                const int *cr = cl.map_shared_rank(counts, r);
                for (int jj = 0; jj < j; ++jj) before += cr[jj];
                if (r < rank && j < NBUCKET) lower += cr[j];
            }
        }
        base_b[j] = before + lower;
        if (rank == 0) a.col_off[(size_t)p * (NBUCKET + 1) + j] = q0 + before;
    }
    if (rank == 0 && tid == 0) {
        int nc = 0;
        if (C == 1) nc = ncol_sh;
        else {
            cg::cluster_group cl = cg::this_cluster();
            for (int r = 0; r < C; ++r) nc = max(nc, *cl.map_shared_rank(&pub_ncol, r));
        }
        a.part_ncol[p] = nc;
        a.part_rounds[p] = rounds;
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < m0; base += T) {
        const int v = base + tid;
        bool valid = v < m0;
        const int k = valid ? item(v) : 0;
        int bucket = NBUCKET;
        if (valid) bucket = 2 * a.p_colour[q0 + k] + ((int)(key[k] >> 62) & 1);
        unsigned peers = __match_any_sync(0xffffffffu, bucket);
        int lrank = __popc(peers & lt);
        if (valid && lrank == 0) wcnt[warp][bucket] = (uint8_t)__popc(peers);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][bucket];
            a.pair_of_row[q0 + base_b[bucket] + running[bucket] + pre + lrank] = q0 + k;
        }
        __syncthreads();
        for (int j = tid; j < NBUCKET; j += T) {
            int add = 0;
            for (int w = 0; w < COLOUR_WARPS; ++w) { add += wcnt[w][j]; wcnt[w][j] = 0; }
            running[j] += add;
        }
        __syncthreads();
    }
    // no CTA may leave while another can still reach its shared memory
    csync<C>();
}

template <int C>
__global__ void __launch_bounds__(COLOUR_THREADS) k_colour(ColourArgs a) {
    extern __shared__ unsigned long long dyn_smem[];
    __shared__ ColourShared sh;
    const int rank = C == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int p = a.order ? (int)a.order[blockIdx.x / C] : (int)(blockIdx.x / C);
    const int nb = a.part_bstart[p + 1] - a.part_bstart[p];
    const int per = (nb + C - 1) / C;
    if (per <= a.smem_slots) {
        unsigned long long *mx = dyn_smem, *u = dyn_smem + per;
        if (C == 1) {
            ColourPtrs S{mx, u};
            colour_worker<1>(a, S, sh, p, 0, per);
        } else {
            ColourSlots<C> S{(uint32_t)__cvta_generic_to_shared(mx), (uint32_t)__cvta_generic_to_shared(u), per};
            colour_worker<C>(a, S, sh, p, rank, per);
        }
    } else if (rank == 0) {
        unsigned long long *mx = a.scratch + 2 * (size_t)a.part_bstart[p];
        ColourPtrs S{mx, mx + nb};
        colour_worker<1>(a, S, sh, p, 0, nb);
    }
}

// ---------------------------------------------------------------------------
// Row records in colour order (the solver forms t1, t2, k_n, k_t and the
// joint k's itself).  Contacts (sphere-sphere or sphere-plane):
//   r0 = (n, slot_b)  r1 = (r_a, r_b, target_n, slot_a)  r3 = (1/m_a, 1/m_b, 1/I_a, 1/I_b)
//   and the impulse record (lambda_n, lambda_t1, lambda_t2, k_n); for a launch
//   with the masses in shared memory r0 = (n, k_t) and r1 = (r_a, r_b,
//   target_n, slot_a | slot_b << 16) with 16-bit slot codes
// Ball joints (rows along the world axes):
//   r0 = (r_A, target_x)  r1 = (r_B, target_y)  r2 = (target_z, 0, slot_a, slot_b)  r3 as for contacts
// A slot word holds the bits of the solver's slot code of a worker slot s:
// rank << 24 | i, with rank = s / per the CTA of the worker's group that
// holds s (per = ceil(nb / C), C the worker's CTAs in the solve plan) and i
// = s - rank per; a static end (or a body not active in this worker) gets
// the zero slot i = per of the CTA that owns the row (the one holding its
// first dynamic body).
// with r_A, r_B the pivot offsets from each body's centre in the world frame.
// ---------------------------------------------------------------------------

// the two slot words of a row (see above), and both as 16-bit codes (rank <<
// 13 | i) packed in one word for a launch with the masses in shared memory;
// a worker of 2^24 bodies or more, or a packed CTA of 8192 slots or more, is
// a capacity error
struct SlotWords { float a, b, packed; };
__device__ __forceinline__ SlotWords slot_words(const RowArgs &a, int p, int2 sl, bool pack) {
    const int nb = a.part_bstart[p + 1] - a.part_bstart[p];
    const int C = max(1, a.solve_C[p]);
    const int per = max(1, (nb + C - 1) / C);
    if (per >= (1 << 24) - 1 || (pack && per >= (1 << 13))) atomicCAS(a.status, DEV_OK, DEV_ERR_SLOTS);
    const int own = sl.x >= 0 ? sl.x / per : max(sl.y, 0) / per;
    auto code = [&](int s, int shift) {
        return s >= 0 ? ((uint32_t)(s / per) << shift | (uint32_t)(s % per)) : ((uint32_t)own << shift | (uint32_t)per);
    };
    const uint32_t p16 = (code(sl.x, 13) & 0xffffu) | (code(sl.y, 13) & 0xffffu) << 16;
    return SlotWords{__uint_as_float(code(sl.x, 24)), __uint_as_float(code(sl.y, 24)), __uint_as_float(p16)};
}

__device__ __forceinline__ bool body_is_box(const float4 *half, int b) {
    if (!half || b < 0) return false;
    const float4 h = half[b];
    return h.x > 0.f || h.y > 0.f || h.z > 0.f;
}

// I^-1 v for body b: a box's R diag(1/I) R^T (R from its blended
// orientation), a sphere's isotropic 1/I
__device__ float3 inv_inertia_times(const RowArgs &a, int b, float3 v) {
    if (!body_is_box(a.half, b)) {
        const float ii = a.st[4 * b + 3].w;
        return make_float3(ii * v.x, ii * v.y, ii * v.z);
    }
    const float4 q = a.st[4 * b + 1], d = a.iib[b];
    const float3 qc = make_float3(-q.y, -q.z, -q.w);                // conjugate: world -> body
    const float3 lb = quat_rotate(make_float4(q.x, qc.x, qc.y, qc.z), v);
    return quat_rotate(q, make_float3(d.x * lb.x, d.y * lb.y, d.z * lb.z));
}

// one full row (see FULL_ROW_WORDS): lever arms rA, rB (world), ends ea, eb
// (-1: static or not in this worker), directions dir[3], targets tg[3]
__device__ void write_full_row(const RowArgs &a, int r, int ea, int eb, float3 rA, float3 rB, const float3 *dir,
                               const float *tg) {
    float4 *F = a.rfull + (size_t)r * FULL_ROW_WORDS;
    const float imA = ea >= 0 ? a.st[4 * ea + 2].w : 0.f, imB = eb >= 0 ? a.st[4 * eb + 2].w : 0.f;
    for (int i = 0; i < 3; ++i) {
        const float3 d = dir[i];
        const float3 jA = make_float3(rA.y * d.z - rA.z * d.y, rA.z * d.x - rA.x * d.z, rA.x * d.y - rA.y * d.x);
        const float3 jB = make_float3(rB.y * d.z - rB.z * d.y, rB.z * d.x - rB.x * d.z, rB.x * d.y - rB.y * d.x);
        const float3 iA = ea >= 0 ? inv_inertia_times(a, ea, jA) : make_float3(0.f, 0.f, 0.f);
        const float3 iB = eb >= 0 ? inv_inertia_times(a, eb, jB) : make_float3(0.f, 0.f, 0.f);
        const float s = (imA + imB) + ((jA.x * iA.x + jA.y * iA.y + jA.z * iA.z) + (jB.x * iB.x + jB.y * iB.y + jB.z * iB.z));
        F[i] = make_float4(d.x, d.y, d.z, tg[i]);
        F[3 + i] = make_float4(jA.x, jA.y, jA.z, s > 0.f ? 1.f / s : 0.f);
        F[6 + i] = make_float4(iA.x, iA.y, iA.z, 0.f);
        F[9 + i] = make_float4(jB.x, jB.y, jB.z, 0.f);
        F[12 + i] = make_float4(iB.x, iB.y, iB.z, 0.f);
    }
    F[15] = make_float4(imA, imB, 0.f, 0.f);
}

__global__ void k_rows(RowArgs a) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.np; r += gridDim.x * blockDim.x) {
        const int k = a.pair_of_row[r];
        const int i = a.ps_cons[k];
        const int2 sl = a.p_slot[k];
        const int scene = a.part_scene[a.ps_part[k]];
        const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[scene];
        const bool pack = a.solve_M && a.solve_M[a.ps_part[k]];   // a launch with the masses in shared memory
        const SlotWords sw = slot_words(a, a.ps_part[k], sl, pack);
        float lam_w = 0.f;   // a plain contact row: k_n (see below)
        if (a.row_full) {
            // a constraint with a box end: the full row, plus the slots in the
            // plain records (the solver reads its bodies through them)
            const int2 ab = i < a.nc ? a.c_ab[i] : a.jab[i - a.nc];
            const bool full = body_is_box(a.half, ab.x) || (ab.y < a.n && body_is_box(a.half, ab.y));
            a.row_full[r] = full ? 1 : 0;
            if (full) {
                const int ea = sl.x >= 0 ? ab.x : -1, eb = sl.y >= 0 ? ab.y : -1;
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                float3 dir[3], rA = make_float3(0.f, 0.f, 0.f), rB = rA;
                float tg[3];
                if (i < a.nc) {
                    const float4 nphi = a.c_n[i], t1 = a.c_t1[i], p = a.c_p[i];
                    dir[0] = make_float3(nphi.x, nphi.y, nphi.z);
                    dir[1] = make_float3(t1.x, t1.y, t1.z);
                    dir[2] = make_float3(dir[0].y * dir[1].z - dir[0].z * dir[1].y, dir[0].z * dir[1].x - dir[0].x * dir[1].z,
                                         dir[0].x * dir[1].y - dir[0].y * dir[1].x);
                    const float4 xa = a.st[4 * ab.x];
                    rA = make_float3(p.x - xa.x, p.y - xa.y, p.z - xa.z);
                    if (ab.y < a.n) {
                        const float4 xb = a.st[4 * ab.y];
                        rB = make_float3(p.x - xb.x, p.y - xb.y, p.z - xb.z);
                    }
                    const float phi = nphi.w;
                    tg[0] = phi > 0.f ? -phi / h : a.erp * fmaxf(-phi - a.slop, 0.f) / h;
                    tg[1] = tg[2] = 0.f;
                    a.r0[r] = make_float4(0.f, 0.f, 0.f, pack ? 0.f : sw.b);
                    a.r1[r] = make_float4(0.f, 0.f, 0.f, pack ? sw.packed : sw.a);
                    a.r3[r] = z;
                } else {
                    const int j = i - a.nc;
                    const float4 anA = a.janc[2 * j], anB = a.janc[2 * j + 1];
                    float3 xA, xB;
                    if (ab.x >= 0) {
                        const float4 x = a.st[4 * ab.x], q = a.st[4 * ab.x + 1];
                        rA = quat_rotate(q, make_float3(anA.x, anA.y, anA.z));
                        xA = make_float3(x.x, x.y, x.z);
                    } else {
                        xA = make_float3(anA.x, anA.y, anA.z);
                    }
                    if (ab.y >= 0) {
                        const float4 x = a.st[4 * ab.y], q = a.st[4 * ab.y + 1];
                        rB = quat_rotate(q, make_float3(anB.x, anB.y, anB.z));
                        xB = make_float3(x.x, x.y, x.z);
                    } else {
                        xB = make_float3(anB.x, anB.y, anB.z);
                    }
                    const float g = -a.erp / h;
                    tg[0] = g * ((xB.x - xA.x) + (rB.x - rA.x));
                    tg[1] = g * ((xB.y - xA.y) + (rB.y - rA.y));
                    tg[2] = g * ((xB.z - xA.z) + (rB.z - rA.z));
                    dir[0] = make_float3(1.f, 0.f, 0.f);
                    dir[1] = make_float3(0.f, 1.f, 0.f);
                    dir[2] = make_float3(0.f, 0.f, 1.f);
                    a.r0[r] = z;
                    a.r1[r] = z;
                    a.r2[r] = make_float4(0.f, 0.f, sw.a, sw.b);
                    a.r3[r] = z;
                }
                write_full_row(a, r, ea, eb, rA, rB, dir, tg);
                a.rpair[r] = k;
                a.rlam[r] = a.p_lam0[k];
                continue;
            }
        }
        if (i < a.nc) {
            const int2 ab = a.c_ab[i];
            const float4 nphi = a.c_n[i];
            const float4 sa = a.st[4 * ab.x + 2], wa = a.st[4 * ab.x + 3], pa = a.st[4 * ab.x];
            float ima = sl.x >= 0 ? sa.w : 0.f, iia = sl.x >= 0 ? wa.w : 0.f;
            float ra = pa.w, rb = 0.f, imb = 0.f, iib = 0.f;
            if (ab.y < a.n) {
                rb = a.st[4 * ab.y].w;
                if (sl.y >= 0) { imb = a.st[4 * ab.y + 2].w; iib = a.st[4 * ab.y + 3].w; }
            }
            float phi = nphi.w;
            float target = phi > 0.f ? -phi / h : a.erp * fmaxf(-phi - a.slop, 0.f) / h;
            if (pack) {
                // k_t with the solver's operations (contact_kt)
                const float kt = __frcp_rn(fmaf(iib, __fmul_rn(rb, rb), fmaf(iia, __fmul_rn(ra, ra), __fadd_rn(ima, imb))));
                a.r0[r] = make_float4(nphi.x, nphi.y, nphi.z, kt);
                a.r1[r] = make_float4(ra, rb, target, sw.packed);
            } else {
                a.r0[r] = make_float4(nphi.x, nphi.y, nphi.z, sw.b);
                a.r1[r] = make_float4(ra, rb, target, sw.a);
            }
            a.r3[r] = make_float4(ima, imb, iia, iib);
            lam_w = __frcp_rn(ima + imb);   // k_n, in the impulse record's spare lane
        } else {
            const int j = i - a.nc;
            const int2 ab = a.jab[j];
            const float4 anA = a.janc[2 * j], anB = a.janc[2 * j + 1];
            // pivot offsets r and reference points x (a world end: x = its
            // pivot, r = 0).  The joint error (xB - xA) + (rB - rA) keeps the
            // large coordinates in one subtraction of nearby values, which is
            // exact in FP32.
            float3 rA = make_float3(0.f, 0.f, 0.f), rB = rA, xA, xB;
            float ima = 0.f, iia = 0.f, imb = 0.f, iib = 0.f;
            if (ab.x >= 0) {
                float4 x = a.st[4 * ab.x], q = a.st[4 * ab.x + 1];
                rA = quat_rotate(q, make_float3(anA.x, anA.y, anA.z));
                xA = make_float3(x.x, x.y, x.z);
                if (sl.x >= 0) { ima = a.st[4 * ab.x + 2].w; iia = a.st[4 * ab.x + 3].w; }
            } else {
                xA = make_float3(anA.x, anA.y, anA.z);
            }
            if (ab.y >= 0) {
                float4 x = a.st[4 * ab.y], q = a.st[4 * ab.y + 1];
                rB = quat_rotate(q, make_float3(anB.x, anB.y, anB.z));
                xB = make_float3(x.x, x.y, x.z);
                if (sl.y >= 0) { imb = a.st[4 * ab.y + 2].w; iib = a.st[4 * ab.y + 3].w; }
            } else {
                xB = make_float3(anB.x, anB.y, anB.z);
            }
            float3 err = make_float3((xB.x - xA.x) + (rB.x - rA.x), (xB.y - xA.y) + (rB.y - rA.y),
                                     (xB.z - xA.z) + (rB.z - rA.z));
            float g = -a.erp / h;
            a.r0[r] = make_float4(rA.x, rA.y, rA.z, g * err.x);
            a.r1[r] = make_float4(rB.x, rB.y, rB.z, g * err.y);
            a.r2[r] = make_float4(g * err.z, 0.f, sw.a, sw.b);
            a.r3[r] = make_float4(ima, imb, iia, iib);
        }
        a.rpair[r] = k;
        const float4 l0 = a.p_lam0[k];
        a.rlam[r] = make_float4(l0.x, l0.y, l0.z, lam_w);
    }
}

}  // namespace

void launch_entry_count(const MemberArgs &a, cudaStream_t s) {
    k_entry_count<<<grid1d(a.n, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}
void launch_entry_fill(const MemberArgs &a, cudaStream_t s) {
    k_entry_fill<<<grid1d(a.n, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}
void launch_entry_slot(const MemberArgs &a, int ne, cudaStream_t s) {
    if (!ne) return;
    k_entry_slot<<<grid1d(ne, 256), 256, 0, s>>>(a, ne);
    note_launch();
    CK(cudaGetLastError());
}
void launch_cons_count(const MemberArgs &a, cudaStream_t s) {
    if (a.nc + a.nj == 0) return;
    k_cons_count<<<grid1d(a.nc + a.nj, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}
void launch_pair_fill(const MemberArgs &a, cudaStream_t s) {
    if (a.nc + a.nj == 0) return;
    k_pair_fill<<<grid1d(a.nc + a.nj, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}
void launch_pair_gather(const MemberArgs &a, const uint32_t *order, int np, cudaStream_t s) {
    if (!np) return;
    k_pair_gather<<<grid1d(np, 256), 256, 0, s>>>(a, order, np);
    note_launch();
    CK(cudaGetLastError());
}
void launch_pair_setup(const MemberArgs &a, const WarmArgs &w, int np, cudaStream_t s) {
    if (!np) return;
    k_pair_setup<<<grid1d(np, 256), 256, 0, s>>>(a, w, np);
    note_launch();
    CK(cudaGetLastError());
}

void launch_row_owner(int P, const int *part_bstart, const int *part_ncol, const int *solve_C,
                      const int *off_in, const int *pair_of_row, const int2 *p_slot,
                      uint8_t *owner_of_row, int *pair_of_row_out, int *off_out, cudaStream_t s) {
    if (P <= 0) return;
    k_row_owner<<<dim3(P, OVL_MAX_COLOURS), OWNER_THREADS, 0, s>>>(P, part_bstart, part_ncol, solve_C, off_in,
                                                                   pair_of_row, p_slot, owner_of_row,
                                                                   pair_of_row_out, off_out);
    note_launch();
    CK(cudaGetLastError());
}

void launch_worker_cost_keys(const int *part_pstart, int P, uint32_t *keys, uint32_t *vals,
                             cudaStream_t s) {
    if (P <= 0) return;
    k_worker_cost_keys<<<grid1d(P, 256), 256, 0, s>>>(part_pstart, P, keys, vals);
    note_launch();
    CK(cudaGetLastError());
}
template <int C>
static void launch_colour_c(const ColourArgs &a, cudaStream_t s) {
    size_t smem = (size_t)a.smem_slots * 2 * sizeof(unsigned long long);
    CK(cudaFuncSetAttribute(k_colour<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_parts * C);
    cfg.blockDim = dim3(COLOUR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, k_colour<C>, a));
    note_launch();
}

// largest static shared memory of the colouring kernels (the per-warp bucket
// counts dominate); the dynamic slot arrays get what is left of the opt-in limit
int colour_static_smem() {
    static int bytes = -1;
    if (bytes < 0) {
        int mx = 0;
        cudaFuncAttributes fa;
        auto take = [&](const void *f) { CK(cudaFuncGetAttributes(&fa, f)); mx = std::max(mx, (int)fa.sharedSizeBytes); };
        take((const void *)k_colour<1>); take((const void *)k_colour<2>); take((const void *)k_colour<3>);
        take((const void *)k_colour<4>); take((const void *)k_colour<6>); take((const void *)k_colour<8>);
        bytes = mx;
    }
    return bytes;
}

void launch_colour(const ColourArgs &a, int cluster, cudaStream_t s) {
    if (!a.n_parts) return;
    switch (cluster) {
        case 8: launch_colour_c<8>(a, s); break;
        case 6: launch_colour_c<6>(a, s); break;
        case 4: launch_colour_c<4>(a, s); break;
        case 3: launch_colour_c<3>(a, s); break;
        case 2: launch_colour_c<2>(a, s); break;
        default: launch_colour_c<1>(a, s); break;
    }
    CK(cudaGetLastError());
}

void launch_rows(const RowArgs &a, cudaStream_t s) {
    if (!a.np) return;
    k_rows<<<grid1d(a.np, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
