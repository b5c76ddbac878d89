// host_alg.cpp -- the sequential, greedy membership algorithms of the method,
// run on the host CPU: ASSIGNTOOVERLAPSET / GROWOVERLAP (Algorithms 2-3,
// Section 5.1) at setup and LOADBALANCE / BRIDGE (Algorithms 6-7, Section 5.4)
// once per step.  Their results depend on the order of the contacts and on
// live worker loads, so they are run exactly in the paper's sequence.
#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "common.cuh"

namespace ovl {

namespace {

inline int popcount(uint64_t x) { return __builtin_popcountll(x); }

// Live load per global worker plus the activate / deactivate primitives of
// Table 1.  The load is |P_w|, or with contact counts deg the sum of
// 1 + deg[b] over the worker's active bodies.  Workers and bodies of
// different scenes are disjoint index ranges, so one instance may be used by
// several threads that each touch only their own scenes.
class Membership {
  public:
    Membership(const HostScene &sc, uint64_t *mask) : sc_(sc), mask_(mask), load_(sc.n_parts, 0) {}
    Membership(const HostScene &sc, uint64_t *mask, const int *loads, const int *deg)
        : sc_(sc), mask_(mask), deg_(deg), load_(loads, loads + sc.n_parts) {}
    // |P_w| of the workers of scenes [s0, s1) from the masks
    void count(int s0, int s1) {
        for (int b = sc_.body_base[s0]; b < sc_.body_base[s1]; ++b) {
            uint64_t m = mask_[b];
            int base = sc_.part_base[sc_.sob[b]];
            while (m) {
                load_[base + __builtin_ctzll(m)] += weight(b);
                m &= m - 1;
            }
        }
    }
    uint64_t W(int b) const { return mask_[b]; }
    const uint64_t *mask_ptr() const { return mask_; }
    void activate(uint64_t workers, int b) {
        uint64_t add = workers & ~mask_[b];
        int base = sc_.part_base[sc_.sob[b]];
        for (uint64_t m = add; m; m &= m - 1) load_[base + __builtin_ctzll(m)] += weight(b);
        mask_[b] |= add;
    }
    void deactivate(uint64_t workers, int b) {
        uint64_t rem = workers & mask_[b];
        int base = sc_.part_base[sc_.sob[b]];
        for (uint64_t m = rem; m; m &= m - 1) load_[base + __builtin_ctzll(m)] -= weight(b);
        mask_[b] &= ~rem;
    }
    // <W>: active bodies (or their weights) summed over the workers of W (Table 1)
    int64_t load(uint64_t workers, int scene) const {
        int64_t s = 0;
        int base = sc_.part_base[scene];
        for (uint64_t m = workers; m; m &= m - 1) s += load_[base + __builtin_ctzll(m)];
        return s;
    }
    // worker of W with the smallest load, lowest index on ties
    int least_loaded(uint64_t workers, int scene) const {
        int base = sc_.part_base[scene];
        int best = -1;
        int64_t best_load = 0;
        for (uint64_t m = workers; m; m &= m - 1) {
            int w = __builtin_ctzll(m);
            if (best < 0 || load_[base + w] < best_load) {
                best = w;
                best_load = load_[base + w];
            }
        }
        return best;
    }

  private:
    int64_t weight(int b) const { return deg_ ? 1 + (int64_t)deg_[b] : 1; }
    const HostScene &sc_;
    uint64_t *mask_;
    const int *deg_ = nullptr;
    std::vector<int64_t> load_;
};

// vertices within `depth` hops of root (root first), over a CSR graph whose
// vertices lie in [lo, lo + n) (one scene: edges never leave it); the
// stamps live in a workspace that outlasts the call
class Ball {
  public:
    Ball(BallWorkspace &w, int n, int lo = 0) : w_(w), lo_(lo) {
        if ((int)w_.seen.size() < n) {
            w_.seen.assign(n, 0);
            w_.epoch = 0;
        }
    }
    const std::vector<int> &collect(const int *row_ptr, const int *col, int root, int depth) {
        if (++w_.epoch == 0x7fffffff) {
            std::fill(w_.seen.begin(), w_.seen.end(), 0);
            w_.epoch = 1;
        }
        const int ep = w_.epoch;
        std::vector<int> &out = w_.out;
        int *seen = w_.seen.data() - lo_;
        out.clear();
        out.push_back(root);
        seen[root] = ep;
        // level by level: [lvl0, lvl1) holds the vertices at distance d
        size_t lvl0 = 0, lvl1 = 1;
        for (int d = 0; d < depth && lvl0 < lvl1; ++d) {
            for (size_t i = lvl0; i < lvl1; ++i) {
                const int u = out[i];
                for (int k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
                    const int v = col[k];
                    if (seen[v] == ep) continue;
                    seen[v] = ep;
                    out.push_back(v);
                }
            }
            lvl0 = lvl1;
            lvl1 = out.size();
        }
        return out;
    }
    void rebase(int lo) { lo_ = lo; }

  private:
    BallWorkspace &w_;
    int lo_;
};

}  // namespace

// Algorithms 2 and 3 over the joints in index order.  The constraint graph
// here is the articulated structure: joints between two dynamic bodies.
void host_assign_overlap(const HostScene &sc, std::vector<uint64_t> &mask) {
    const int n = sc.n;
    const int nj = (int)sc.jab.size() / 2;
    auto dyn = [&](int b) { return b >= 0 && b < n && sc.inv_mass[b] > 0.0f; };
    std::vector<int> deg(n + 1, 0);
    for (int j = 0; j < nj; ++j) {
        int a = sc.jab[2 * j], b = sc.jab[2 * j + 1];
        if (dyn(a) && dyn(b) && a != b) { ++deg[a]; ++deg[b]; }
    }
    std::vector<int> row_ptr(n + 1, 0);
    for (int i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i];
    std::vector<int> col(row_ptr[n]);
    std::vector<int> fill(row_ptr.begin(), row_ptr.end() - 1);
    for (int j = 0; j < nj; ++j) {
        int a = sc.jab[2 * j], b = sc.jab[2 * j + 1];
        if (dyn(a) && dyn(b) && a != b) { col[fill[a]++] = b; col[fill[b]++] = a; }
    }
    // sorted, duplicate-free neighbour lists (the BFS result is a set anyway)
    for (int i = 0; i < n; ++i) {
        auto first = col.begin() + row_ptr[i], last = col.begin() + row_ptr[i + 1];
        std::sort(first, last);
    }
    Membership mem(sc, mask.data());
    mem.count(0, sc.ns);
    BallWorkspace bw;
    Ball ball(bw, n);
    auto grow = [&](int root, int gamma, uint64_t Wr) {      // Algorithm 3
        const std::vector<int> &N = ball.collect(row_ptr.data(), col.data(), root, gamma);
        for (int b : N)
            if (popcount(mem.W(b)) < 2) mem.activate(Wr & ~mem.W(b), b);
    };
    for (int j = 0; j < nj; ++j) {
        int A = sc.jab[2 * j], B = sc.jab[2 * j + 1];
        if (!dyn(A) || !dyn(B) || A == B) continue;
        uint64_t WA = mem.W(A), WB = mem.W(B);
        if (popcount(WA) != 1 || popcount(WB) != 1 || WA == WB) continue;   // joint across workers
        int gamma = sc.scene_gamma[sc.sob[A]];
        mem.activate(mem.W(B), A);
        grow(A, gamma, mem.W(A) | mem.W(B));
        mem.activate(mem.W(A), B);
        grow(B, gamma, mem.W(A) | mem.W(B));
    }
}

namespace {

// Algorithm 6 over candidates [i0, i1), all of scenes [s0, s1)
void load_balance_range(const HostScene &sc, Membership &mem, const int2 *ab, int64_t i0, int64_t i1,
                        int s0, int s1, const int *row_ptr, const int *col, bool do_activate,
                        bool do_deactivate, BallWorkspace &bw, const int *ball_start, const int *ball_vtx) {
    if (i0 == i1) return;
    int widest = 0;
    for (int s = s0; s < s1; ++s) widest = std::max(widest, sc.body_base[s + 1] - sc.body_base[s]);
    Ball ball(bw, widest, sc.body_base[s0]);
    int ball_scene = -1;
    auto bridge = [&](int b) {                                  // Algorithm 7
        // the union of the neighbours' workers has more than one worker:
        // decided as soon as two different workers have been seen
        uint64_t u = 0;
        for (int k = row_ptr[b]; k < row_ptr[b + 1]; ++k) {
            u |= mem.W(col[k]);
            if (u & (u - 1)) return true;
        }
        return false;
    };
    constexpr int64_t kAhead = 16;   // candidates between a prefetch and its use
    constexpr int64_t kBallAhead = 4;   // the same for the masks of balls found beforehand
    for (int64_t i = i0; i < i1; ++i) {
        if (ball_start && i + kBallAhead < i1) {
            // either end may become the root: fetch the masks of both balls
            const int2 e = ab[i + kBallAhead];
            for (int k = ball_start[e.x]; k < ball_start[e.x + 1]; ++k) __builtin_prefetch(mem.mask_ptr() + ball_vtx[k]);
            for (int k = ball_start[e.y]; k < ball_start[e.y + 1]; ++k) __builtin_prefetch(mem.mask_ptr() + ball_vtx[k]);
        }
        if (i + kAhead < i1) {
            // the second body of a contact is a random index: fetch its mask
            // and adjacency range while earlier candidates are processed
            const int Bn = ab[i + kAhead].y;
            __builtin_prefetch(mem.mask_ptr() + Bn);
            __builtin_prefetch(row_ptr + Bn);
            __builtin_prefetch(sc.sob.data() + ab[i + kAhead].x);
        }
        const int A = ab[i].x, B = ab[i].y;
        const uint64_t WA = mem.W(A), WB = mem.W(B);
        const int scene = sc.sob[A];
        if ((WA & WB) == 0) {                                   // activation branch
            if (!do_activate) continue;
            int root;
            if (mem.load(WA, scene) <= mem.load(WB, scene)) {   // ties: B joins W_A
                mem.activate(WA, B);
                root = B;
            } else {
                mem.activate(WB, A);
                root = A;
            }
            if (ball_start && ball_start[root + 1] > ball_start[root]) {
                // the gamma-ball found beforehand (the same vertex set)
                for (int k = ball_start[root]; k < ball_start[root + 1]; ++k) {
                    const int v = ball_vtx[k];
                    mem.activate((WA | WB) & ~mem.W(v), v);
                }
                continue;
            }
            if (scene != ball_scene) { ball.rebase(sc.body_base[scene]); ball_scene = scene; }
            const std::vector<int> &N =
                ball.collect(row_ptr, col, root, sc.scene_gamma[scene]);   // gamma-ball
            for (int v : N) mem.activate((WA | WB) & ~mem.W(v), v);
            continue;
        }
        if (!do_deactivate) continue;
        const int pa = popcount(WA), pb = popcount(WB);
        if (pa > 1 && pb == 1 && !bridge(A)) {
            mem.deactivate(WA & ~WB, A);
        } else if (pb > 1 && pa == 1 && !bridge(B)) {
            mem.deactivate(WB & ~WA, B);
        } else if (WA == WB) {
            uint64_t keep = uint64_t(1) << mem.least_loaded(WA, scene);   // ties -> lowest
            mem.deactivate(WA & ~keep, A);
            mem.deactivate(WB & ~keep, B);
        }
    }
}

}  // namespace

// Algorithm 6 over contacts between dynamic bodies, in canonical order.
// Contacts of one scene are contiguous in that order and touch only that
// scene's masks and worker loads, so runs of whole scenes go to up to
// `threads` host threads; the result is the sequential one.
void host_load_balance(const HostScene &sc, uint64_t *mask, const int *loads, const int *deg, int64_t nc,
                       const int2 *ab, const int *row_ptr, const int *col, bool do_activate,
                       bool do_deactivate, std::vector<BallWorkspace> &ws, const int *ball_start,
                       const int *ball_vtx) {
    if (nc == 0 || (!do_activate && !do_deactivate) || ws.empty()) return;
    const int threads = (int)ws.size();
    Membership mem(sc, mask, loads, deg);
    // candidate range of every scene
    std::vector<int64_t> first(sc.ns + 1, nc);
    for (int64_t i = nc - 1; i >= 0; --i) first[sc.sob[ab[i].x]] = i;
    for (int s = sc.ns - 1; s >= 0; --s) first[s] = std::min(first[s], first[s + 1]);
    // chunks of whole scenes with about equal candidates plus bodies
    const int T = std::max(1, std::min(threads, sc.ns));
    std::vector<int> cut{0};
    const double per = (double)(nc + sc.n) / T;
    double acc = 0.0;
    for (int s = 0; s < sc.ns; ++s) {
        acc += (double)(first[s + 1] - first[s]) + (sc.body_base[s + 1] - sc.body_base[s]);
        if (acc >= per * (double)cut.size() && (int)cut.size() < T && s + 1 < sc.ns) cut.push_back(s + 1);
    }
    cut.push_back(sc.ns);
    auto run = [&](size_t k) {
        const int s0 = cut[k], s1 = cut[k + 1];
        load_balance_range(sc, mem, ab, first[s0], first[s1], s0, s1, row_ptr, col, do_activate,
                           do_deactivate, ws[k], ball_start, ball_vtx);
    };
    if (cut.size() == 2) {
        run(0);
        return;
    }
    std::vector<std::thread> pool;
    for (size_t k = 1; k + 1 < cut.size(); ++k) pool.emplace_back(run, k);
    run(0);
    for (auto &t : pool) t.join();
}

}  // namespace ovl
