// k_member.cu -- who solves what (Section 4, Eq 9-10): membership entries
// (body, worker), every worker's body list and local slots, the
// (worker, constraint) pairs with their warm-start impulses, the per-worker
// colouring that orders the Gauss-Seidel sweep, and the colour-ordered row
// records the solver streams.
#include "common.cuh"
#include "kernels.cuh"

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

__global__ void k_pair_setup(MemberArgs a, WarmArgs ws, int np) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        int i = a.ps_cons[k], p = a.ps_part[k];
        int scene = cons_scene(i, a.nc, a.c_ab, a.sob, a.joint_scene);
        int w = p - a.part_base[scene];
        int2 e;
        uint64_t key;
        if (i < a.nc) {
            e = a.c_ab[i];
            key = ((uint64_t)(uint32_t)e.x << 32) | (uint32_t)e.y;
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

constexpr int COLOUR_THREADS = 512;
constexpr int COLOUR_WARPS = COLOUR_THREADS / 32;
constexpr int NBUCKET = 2 * OVL_MAX_COLOURS;

__global__ void __launch_bounds__(COLOUR_THREADS) k_colour(ColourArgs a) {
    extern __shared__ unsigned long long dyn_smem[];
    __shared__ int n_cur, n_next, rounds_left, ncol_sh;
    __shared__ int counts[NBUCKET + 1];
    __shared__ int running[NBUCKET];
    __shared__ int wcnt[COLOUR_WARPS][NBUCKET];
    const int p = blockIdx.x;
    const int tid = threadIdx.x;
    const int b0 = a.part_bstart[p], nb = a.part_bstart[p + 1] - b0;
    const int q0 = a.part_pstart[p], nq = a.part_pstart[p + 1] - q0;
    unsigned long long *slot_max, *used0, *used1;
    if (nb <= a.smem_slots) {
        slot_max = dyn_smem;
    } else {
        slot_max = a.scratch + 3 * (size_t)b0;
    }
    used0 = slot_max + nb;
    used1 = used0 + nb;
    // worklists of uncoloured constraints, ping-pong: (index relative to q0,
    // slot a, slot b) and the priority, read contiguously every round
    int4 *wl_cur = a.worklist + q0, *wl_next = a.worklist2 + q0;
    unsigned long long *pr_cur = a.wprio + q0, *pr_next = a.wprio2 + q0;
    for (int s = tid; s < nb; s += blockDim.x) { used0[s] = 0ull; used1[s] = 0ull; slot_max[s] = 0ull; }
    for (int k = tid; k < nq; k += blockDim.x) {
        int2 sl = a.p_slot[q0 + k];
        wl_cur[k] = make_int4(k, sl.x, sl.y, 0);
        pr_cur[k] = mix64(a.p_key[q0 + k]);
    }
    if (tid == 0) { n_cur = nq; n_next = 0; rounds_left = nq + 2; ncol_sh = 0; }
    __syncthreads();
    while (n_cur > 0 && rounds_left > 0) {
        const int m = n_cur;
        // highest priority among the uncoloured constraints at every slot
        for (int i = tid; i < m; i += blockDim.x) {
            const int4 w = wl_cur[i];
            const unsigned long long pr = pr_cur[i];
            if (w.y >= 0) atomicMax(&slot_max[w.y], pr);
            if (w.z >= 0) atomicMax(&slot_max[w.z], pr);
        }
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) {
            const int4 w = wl_cur[i];
            const unsigned long long pr = pr_cur[i];
            bool ready = (w.y < 0 || slot_max[w.y] == pr) && (w.z < 0 || slot_max[w.z] == pr);
            if (!ready) {
                int o = atomicAdd(&n_next, 1);
                wl_next[o] = w;
                pr_next[o] = pr;
                continue;
            }
            // only this constraint touches its slots in this round
            unsigned long long u0 = 0ull, u1 = 0ull;
            if (w.y >= 0) { u0 |= used0[w.y]; u1 |= used1[w.y]; }
            if (w.z >= 0) { u0 |= used0[w.z]; u1 |= used1[w.z]; }
            int c;
            if (~u0) c = __ffsll((long long)~u0) - 1;
            else if (~u1) c = 64 + __ffsll((long long)~u1) - 1;
            else { c = OVL_MAX_COLOURS - 1; atomicCAS(a.status, DEV_OK, DEV_ERR_COLOURS); }
            a.p_colour[q0 + w.x] = c;
            unsigned long long bit0 = c < 64 ? (1ull << c) : 0ull, bit1 = c >= 64 ? (1ull << (c - 64)) : 0ull;
            if (w.y >= 0) { used0[w.y] |= bit0; used1[w.y] |= bit1; }
            if (w.z >= 0) { used0[w.z] |= bit0; used1[w.z] |= bit1; }
            atomicMax(&ncol_sh, c + 1);
        }
        __syncthreads();
        // clear the slot maxima that this round set
        for (int i = tid; i < m; i += blockDim.x) {
            const int4 w = wl_cur[i];
            if (w.y >= 0) slot_max[w.y] = 0ull;
            if (w.z >= 0) slot_max[w.z] = 0ull;
        }
        __syncthreads();
        if (tid == 0) { n_cur = n_next; n_next = 0; --rounds_left; }
        int4 *t = wl_cur; wl_cur = wl_next; wl_next = t;
        unsigned long long *tp = pr_cur; pr_cur = pr_next; pr_next = tp;
        __syncthreads();
    }
    if (tid == 0 && n_cur > 0) atomicCAS(a.status, DEV_OK, DEV_ERR_TIMEOUT);
    // stable counting sort of the worker's constraints by (colour, kind):
    // contacts before joints inside a colour, canonical order kept
    for (int j = tid; j <= NBUCKET; j += blockDim.x) counts[j] = 0;
    for (int j = tid; j < NBUCKET; j += blockDim.x) running[j] = 0;
    for (int j = tid; j < COLOUR_WARPS * NBUCKET; j += blockDim.x) (&wcnt[0][0])[j] = 0;
    __syncthreads();
    for (int k = tid; k < nq; k += blockDim.x) {
        int c = a.p_colour[q0 + k];
        int kind = (int)(a.p_key[q0 + k] >> 62) & 1;
        atomicAdd(&counts[2 * c + kind], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int j = 0; j <= NBUCKET; ++j) {
            int v = j < NBUCKET ? counts[j] : 0;
            counts[j] = acc;
            acc += v;
        }
        a.part_ncol[p] = ncol_sh;
    }
    __syncthreads();
    int *off = a.col_off + (size_t)p * (NBUCKET + 1);
    for (int j = tid; j <= NBUCKET; j += blockDim.x) off[j] = q0 + counts[j];
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < nq; base += blockDim.x) {
        int k = base + tid;
        bool valid = k < nq;
        int bucket = NBUCKET;
        if (valid) bucket = 2 * a.p_colour[q0 + k] + ((int)(a.p_key[q0 + k] >> 62) & 1);
        unsigned peers = __match_any_sync(0xffffffffu, bucket);
        int lrank = __popc(peers & lt);
        if (valid && lrank == 0) wcnt[warp][bucket] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][bucket];
            int row = q0 + counts[bucket] + running[bucket] + pre + lrank;
            a.pair_of_row[row] = q0 + k;
        }
        __syncthreads();
        for (int j = tid; j < NBUCKET; j += blockDim.x) {
            int add = 0;
            for (int w = 0; w < COLOUR_WARPS; ++w) { add += wcnt[w][j]; wcnt[w][j] = 0; }
            running[j] += add;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row records in colour order.  Contacts (sphere-sphere or sphere-plane):
//   r0 = (n, k_n)  r1 = (t1, k_t)  r2 = (r_a, r_b, target_n, mu)  r3 = (slot_a, slot_b, pair, 0)
// Ball joints (rows along the world axes):
//   r0 = (r_A, target_x)  r1 = (r_B, target_y)  r2 = (k_x, k_y, k_z, target_z)  r3 = (.., .., pair, 1)
// with r_A, r_B the pivot offsets from each body's centre in the world frame.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 quat_rotate(float4 q, float3 v) {
    // v + 2 w (u x v) + 2 u x (u x v), q = (w, u)
    float3 u = make_float3(q.y, q.z, q.w);
    float3 t = make_float3(2.f * (u.y * v.z - u.z * v.y), 2.f * (u.z * v.x - u.x * v.z),
                           2.f * (u.x * v.y - u.y * v.x));
    return make_float3(v.x + q.x * t.x + (u.y * t.z - u.z * t.y),
                       v.y + q.x * t.y + (u.z * t.x - u.x * t.z),
                       v.z + q.x * t.z + (u.x * t.y - u.y * t.x));
}

// two 16-bit worker slots in one word (0xffff: static end)
__device__ __forceinline__ int pack_slots(int2 sl, int *status) {
    if (sl.x >= 0xffff || sl.y >= 0xffff) atomicCAS(status, DEV_OK, DEV_ERR_CAPACITY);
    unsigned a = sl.x < 0 ? 0xffffu : (unsigned)sl.x & 0xffffu;
    unsigned b = sl.y < 0 ? 0xffffu : (unsigned)sl.y & 0xffffu;
    return (int)(a | (b << 16));
}

__global__ void k_rows(RowArgs a) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.np; r += gridDim.x * blockDim.x) {
        const int k = a.pair_of_row[r];
        const int i = a.ps_cons[k];
        const int2 sl = a.p_slot[k];
        const int scene = a.part_scene[a.ps_part[k]];
        const float h = a.dt_override > 0.f ? a.dt_override : a.scene_dt[scene];
        if (i < a.nc) {
            const int2 ab = a.c_ab[i];
            const float4 nphi = a.c_n[i];
            const float4 t1 = a.c_t1[i];
            const float4 sa = a.st[4 * ab.x + 2], wa = a.st[4 * ab.x + 3], pa = a.st[4 * ab.x];
            float ima = sl.x >= 0 ? sa.w : 0.f, iia = sl.x >= 0 ? wa.w : 0.f;
            float ra = pa.w, rb = 0.f, imb = 0.f, iib = 0.f;
            if (ab.y < a.n) {
                rb = a.st[4 * ab.y].w;
                if (sl.y >= 0) { imb = a.st[4 * ab.y + 2].w; iib = a.st[4 * ab.y + 3].w; }
            }
            float kn = 1.0f / (ima + imb);
            float kt = 1.0f / (ima + imb + iia * ra * ra + iib * rb * rb);
            float phi = nphi.w;
            float target = phi > 0.f ? -phi / h : a.erp * fmaxf(-phi - a.slop, 0.f) / h;
            a.r0[r] = make_float4(nphi.x, nphi.y, nphi.z, kn);
            a.r1[r] = make_float4(t1.x, t1.y, t1.z, kt);
            a.r2[r] = make_float4(ra, rb, target, __int_as_float(pack_slots(sl, a.status)));
            a.r3[r] = make_float4(ima, imb, iia, iib);
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
            a.r2[r] = make_float4(g * err.z, 0.f, 0.f, __int_as_float(pack_slots(sl, a.status)));
            a.r3[r] = make_float4(ima, imb, iia, iib);
        }
        a.rpair[r] = k;
        a.rlam[r] = a.p_lam0[k];
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
void launch_colour(const ColourArgs &a, cudaStream_t s) {
    if (!a.n_parts) return;
    size_t smem = (size_t)a.smem_slots * 3 * sizeof(unsigned long long);
    CK(cudaFuncSetAttribute(k_colour, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_colour<<<a.n_parts, COLOUR_THREADS, smem, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}
void launch_rows(const RowArgs &a, cudaStream_t s) {
    if (!a.np) return;
    k_rows<<<grid1d(a.np, 256), 256, 0, s>>>(a);
    note_launch();
    CK(cudaGetLastError());
}

}  // namespace ovl
