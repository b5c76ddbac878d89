"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: the paper's
worked examples (``tests/golden``), closed-form rigid-body answers, brute force
(Floyd-Warshall, all-pairs contact search, enumeration of MLCP active sets),
a library routine (networkx greedy colouring) or an invariant of the method.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_17261_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 9.81


def _scene(pos, radius, inv_mass, planes=(), sets=None, n_sets=1, joints=None, anchors=None,
           mu=0.5, dt=1.0 / 60.0, flags=1, gamma=0, beta=2, iters=20, lb_deact_every=1):
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    sets = np.zeros(n, np.int32) if sets is None else np.asarray(sets)
    return S._single("t", pos, radius, inv_mass, np.asarray(planes, dtype=np.float64).reshape(-1, 4),
                     mu=mu, dt=dt, flags=flags, gamma=gamma, beta=beta, n_sets=n_sets,
                     set_of_body=sets, joints=joints, anchors=anchors, iters=iters, steps=1,
                     lb_deact_every=lb_deact_every)


def _popc(x):
    return bin(int(x)).count("1")


def _bits(ws):
    m = 0
    for w in ws:
        m |= 1 << w
    return m


# ---------------------------------------------------------------------------
# worked examples printed in the paper
# ---------------------------------------------------------------------------

def test_fig2_overlap_set():
    g = json.load(open(os.path.join(GOLDEN, "fig2_sets.json")))
    n = len(g["A"])
    pos = [[10.0 * i, 0.0, 50.0] for i in range(n)]            # far apart: no contacts
    sc = _scene(pos, np.full(n, 0.5), np.ones(n), planes=[[0, 0, 1, 0]], n_sets=2,
                sets=np.zeros(n))
    sim = O.OracleSim(sc)
    masks = np.zeros(n, np.uint64)
    for b in g["P1"]:
        masks[b - 1] |= np.uint64(1)
    for b in g["P2"]:
        masks[b - 1] |= np.uint64(2)
    sim.set_masks(masks)
    sim.step()
    ent = sim.entries()
    ep = ent["entry_ptr"]
    overlap = [b + 1 for b in range(n) if ep[b + 1] - ep[b] >= 2]
    assert overlap == g["O"]
    # with no constraint edges no worker is met: uniform weights (reading of Alg 5)
    for b in g["O"]:
        w = ent["weight"][ep[b - 1]:ep[b]]
        assert np.allclose(w, [0.5, 0.5])


def test_fig3_chain_articulated_assignment():
    g = json.load(open(os.path.join(GOLDEN, "fig3_chain.json")))
    n = len(g["bodies"])
    joints = np.array(g["joints"]) - 1
    masks = np.array([1 << (g["worker_of_body"][str(b)] - 1) for b in g["bodies"]], dtype=np.uint64)
    sob = np.zeros(n, np.int32)
    for gamma, key in [(0, "gamma0_overlap"), (1, "gamma1_overlap")]:
        out = O.assign_overlap(masks, sob, [2], np.ones(n), joints, [gamma])
        overlap = [b + 1 for b in range(n) if _popc(out[b]) >= 2]
        assert overlap == g[key]
        assert all(_popc(x) >= 1 for x in out)


def test_splitmix64_reference_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    want = [int(x, 16) for x in g["outputs_hex"]]
    got = [int(x) for x in S.SplitMix64(g["seed"]).next_u64(3)]
    assert got == want
    # the oracle's priority hash is the same finaliser applied to a raw state
    gamma = 0x9E3779B97F4A7C15
    assert [O.mix64((k + 1) * gamma) for k in range(3)] == want


# ---------------------------------------------------------------------------
# Algorithm 6 scenarios (Figure 9 (i)-(v), Section 5.4) and Algorithm 7
# ---------------------------------------------------------------------------

def _lb(masks, n_sets, contacts, extra_edges=(), gamma=0, act=True, deact=True):
    masks = np.array(masks, dtype=np.uint64)
    n = masks.shape[0]
    edges = list(contacts) + list(extra_edges)
    rp, col = O.graph(n, np.ones(n), edges if edges else np.zeros((0, 2)))
    return O.load_balance(masks, np.zeros(n, np.int32), [n_sets], rp, col,
                          np.array(contacts, dtype=np.int32).reshape(-1, 2), [gamma], act, deact)


def test_lb_inter_worker_goes_to_lighter_side():
    # (i): A=0 in worker 0 with 3 idle companions, B=1 alone in worker 1:
    # <W_A> = 4 > <W_B> = 1, so A is activated in W_B
    out = _lb([1, 2, 1, 1, 1], 2, [(0, 1)])
    assert list(out) == [3, 2, 1, 1, 1]


def test_lb_tie_activates_b_in_wa():
    # equal loads: the comparison is <=, so B joins W_A
    out = _lb([1, 2], 2, [(0, 1)])
    assert list(out) == [1, 3]


def test_lb_growth_depth():
    # (ii) with growth: A=0 links to C=2 -> D=3 -> E=4 (all worker 0); B=1 in
    # worker 1.  <W_A> = 4 > <W_B> = 1 so root = A; every vertex within 2 hops
    # of A (A, B, C, D) gets W_A u W_B.
    out = _lb([1, 2, 1, 1, 1], 2, [(0, 1)], extra_edges=[(0, 2), (2, 3), (3, 4)], gamma=2)
    assert list(out) == [3, 3, 3, 3, 1]


def test_lb_overlap_not_bridge_is_removed():
    # (iii): B=1 in both workers touches only A=0 (worker 0): not a bridge, so
    # B keeps only W_A
    out = _lb([1, 3], 2, [(0, 1)])
    assert list(out) == [1, 1]


def test_lb_bridge_is_kept():
    # (iv): B=1 in both workers touches A=0 (worker 0) and C=2 (worker 1)
    out = _lb([1, 3, 2], 2, [(0, 1), (1, 2)])
    assert list(out) == [1, 3, 2]
    rp, col = O.graph(3, np.ones(3), [(0, 1), (1, 2)])
    assert O.is_bridge(np.array([1, 3, 2], np.uint64), rp, col, 1)
    assert not O.is_bridge(np.array([1, 3, 1], np.uint64), rp, col, 1)


def test_lb_two_overlap_bodies_keep_least_loaded():
    # (v): A=0, B=1 both in workers {0,1}; worker 0 has 2 more bodies, worker 1
    # one more: counts 4 vs 3 -> keep worker 1 only
    out = _lb([3, 3, 1, 1, 2], 2, [(0, 1)])
    assert list(out) == [2, 2, 1, 1, 2]
    # equal counts: ties go to the lowest worker index
    out = _lb([3, 3, 1, 2], 2, [(0, 1)])
    assert list(out) == [1, 1, 1, 2]


def test_lb_removal_branches_respect_cadence():
    out = _lb([1, 3], 2, [(0, 1)], deact=False)
    assert list(out) == [1, 3]
    out = _lb([1, 2], 2, [(0, 1)], act=False)
    assert list(out) == [1, 2]


# ---------------------------------------------------------------------------
# The contact load (Section 6): <W> sums 1 + contacts over active bodies
# ---------------------------------------------------------------------------

def _lb_w(masks, n_sets, contacts, weights, act=True, deact=True):
    masks = np.array(masks, dtype=np.uint64)
    n = masks.shape[0]
    rp, col = O.graph(n, np.ones(n), list(contacts))
    return O.load_balance(masks, np.zeros(n, np.int32), [n_sets], rp, col,
                          np.array(contacts, dtype=np.int32).reshape(-1, 2), [0], act, deact,
                          weights=np.array(weights, dtype=np.int64))


def test_contact_load_flips_the_activation_side():
    # the case of test_lb_inter_worker_goes_to_lighter_side with B carrying
    # weight 10: <W_A> = 4 <= <W_B> = 10, so now B joins W_A
    out = _lb_w([1, 2, 1, 1, 1], 2, [(0, 1)], [1, 10, 1, 1, 1])
    assert list(out) == [1, 3, 1, 1, 1]
    # unit weights are the body count
    assert list(_lb_w([1, 2, 1, 1, 1], 2, [(0, 1)], [1] * 5)) == [3, 2, 1, 1, 1]


def test_contact_load_is_live():
    # worker 0 = {0, 2} (load 2), worker 1 = {1, 3} (weights 5 + 1 = 6).
    # Contact (0, 1): 2 <= 6, body 1 joins worker 0, whose load becomes 7 --
    # by body 1's weight, not by 1.  Contact (2, 3): 7 > 6, so body 2 joins
    # worker 1.  (Adding 1 instead would give 3 <= 6 and body 3 joining worker 0.)
    out = _lb_w([1, 2, 1, 2], 2, [(0, 1), (2, 3)], [1, 5, 1, 1])
    assert list(out) == [1, 3, 3, 2]


def test_contact_load_least_loaded_keep():
    # the case of test_lb_two_overlap_bodies_keep_least_loaded: by count
    # worker 1 is kept; with body 4 (worker 1 only) weighing 5, worker 0's
    # load 4 is below worker 1's 7 and worker 0 is kept
    out = _lb_w([3, 3, 1, 1, 2], 2, [(0, 1)], [1, 1, 1, 1, 5])
    assert list(out) == [1, 1, 1, 1, 2]


def _corner_scene(extra_w1):
    """Sphere A (worker 0) in the corner of a floor z = 0 and a wall x = 0,
    touching both; sphere B (worker 1) resting on A along the diagonal, clear
    of both planes; free spheres far above: one in worker 0, extra_w1 in
    worker 1.  A's contacts: floor, wall, B (weight 4); B's: A (weight 2)."""
    h = 1.0 / np.sqrt(2.0)
    pos = [(0.5, 5.0, 0.5), (0.5 + h, 5.0, 0.5 + h), (20.0, 5.0, 30.0)]
    sets = [0, 1, 0]
    for k in range(extra_w1):
        pos.append((20.0 + 3.0 * (k + 1), 5.0, 30.0))
        sets.append(1)
    n = len(pos)
    planes = [(0.0, 0.0, 1.0, 0.0), (1.0, 0.0, 0.0, 0.0)]
    return S._single("corner", np.array(pos), np.full(n, 0.5), np.ones(n), planes, mu=0.5,
                     dt=1.0 / 60.0, flags=1, gamma=0, beta=2, n_sets=2, set_of_body=sets,
                     iters=10, steps=1)


def test_contact_load_counts_every_contact_of_the_step():
    # bodies: <W_0> = 2 <= <W_1> = 3, B joins worker 0.  Contacts: <W_0> =
    # 4 + 1 = 5 > <W_1> = 2 + 1 + 1 = 4, A joins worker 1 -- only if both plane
    # contacts of A count (without them A weighs 2 and <W_0> = 3).
    out = {}
    for load in (0, 1):
        sim = O.OracleSim(_corner_scene(2), dict(lb_load=load))
        sim.step()
        out[load] = [int(m) for m in sim.masks()[:2]]
    assert out[0] == [1, 3]
    assert out[1] == [3, 2]


def test_contact_load_counts_the_body_itself():
    # four free spheres in worker 1: <W_0> = 4 + 1 = 5 <= <W_1> = 2 + 4 = 6 and
    # B joins worker 0 -- only with the 1 per body (contacts alone: 3 > 1)
    sim = O.OracleSim(_corner_scene(4), dict(lb_load=1))
    sim.step()
    assert [int(m) for m in sim.masks()[:2]] == [1, 3]


# ---------------------------------------------------------------------------
# Joint violation (Section 6's error measure) and uniform weights (Figure 8)
# ---------------------------------------------------------------------------

def _pair_scene(pos, joints, anchors):
    n = len(pos)
    return S._single("pair", np.array(pos, dtype=np.float64), np.full(n, 0.1), np.ones(n), [],
                     mu=0.5, dt=1.0 / 60.0, flags=0, gamma=0, beta=2, n_sets=1,
                     set_of_body=np.zeros(n, np.int32), joints=joints, anchors=anchors)


def test_joint_error_closed_forms():
    # bodies at (0,0,0) and (2,0,0), pivot halfway: no gap
    sc = _pair_scene([(0, 0, 0), (2, 0, 0)], [(0, 1)], [(1, 0, 0, -1, 0, 0)])
    sim = O.OracleSim(sc)
    assert sim.joint_error() == dict(sum=0.0, max=0.0)
    st = sim.state()
    st[1, 1] += 0.3                                   # B moved sideways: gap 0.3
    sim.set_state(st)
    assert sim.joint_error()["sum"] == pytest.approx(0.3, abs=1e-15)
    st = sim.state()
    st[1, 1] -= 0.3
    c = math.cos(math.pi / 4)
    st[0, 3:7] = (c, 0.0, 0.0, c)                     # A turned 90 degrees about z
    sim.set_state(st)
    # A's pivot moves from (1,0,0) to (0,1,0); B's stays at (1,0,0)
    assert sim.joint_error()["max"] == pytest.approx(math.sqrt(2.0), abs=1e-12)
    # a world end: the world pivot itself
    sc = _pair_scene([(0, 0, 0), (3, 0, 0)], [(-1, 0), (1, -1)],
                     [(-1, 0, 0, -1, 0, 0), (0, 0, 0.5, 3, 0, 0)])
    sim = O.OracleSim(sc)
    e = sim.joint_error()
    assert e["sum"] == pytest.approx(0.5, abs=1e-15) and e["max"] == pytest.approx(0.5, abs=1e-15)


def _weight_chain(weights):
    # six bodies in a jointed row; workers {0}, {0}, {0,1}, {0,1}, {1}, {1}
    pos = [(float(i), 0.0, 5.0) for i in range(6)]
    joints = [(i, i + 1) for i in range(5)]
    anchors = [(0.5, 0, 0, -0.5, 0, 0)] * 5
    n = 6
    sc = S._single("row", np.array(pos), np.full(n, 0.1), np.ones(n), [], mu=0.5, dt=1.0 / 60.0,
                   flags=0, gamma=0, beta=3, n_sets=2, set_of_body=[0, 0, 0, 1, 1, 1],
                   joints=joints, anchors=anchors, lb_activate=0, lb_deact_every=0)
    sim = O.OracleSim(sc, dict(weights=weights))
    sim.set_masks(np.array([1, 1, 3, 3, 2, 2], np.uint64))
    sim.step()
    return sim.entries()


def test_uniform_weights_against_geodesic():
    g, u = _weight_chain(0), _weight_chain(1)
    assert np.array_equal(g["D"], u["D"])
    # body 2: one hop from worker 0's body 1, two from worker 1's body 4
    e2 = slice(int(g["entry_ptr"][2]), int(g["entry_ptr"][3]))
    assert list(g["D"][e2]) == [1, 2]
    np.testing.assert_allclose(g["weight"][e2], [2 / 3, 1 / 3], rtol=0, atol=1e-15)
    np.testing.assert_allclose(u["weight"][e2], [0.5, 0.5], rtol=0, atol=0)
    e3 = slice(int(g["entry_ptr"][3]), int(g["entry_ptr"][4]))
    np.testing.assert_allclose(g["weight"][e3], [1 / 3, 2 / 3], rtol=0, atol=1e-15)
    np.testing.assert_allclose(u["weight"][e3], [0.5, 0.5], rtol=0, atol=0)
    # single-worker bodies weigh 1 either way
    assert u["weight"][0] == 1.0 and u["weight"][-1] == 1.0


# ---------------------------------------------------------------------------
# Geodesic distances and weights (Eq 15-16, Algorithm 5)
# ---------------------------------------------------------------------------

def test_chain_weights_closed_form():
    # 7-body chain, only the middle body shared: equidistant -> (1/2, 1/2)
    n = 7
    edges = [(i, i + 1) for i in range(n - 1)]
    rp, col = O.graph(n, np.ones(n), edges)
    masks = np.array([1, 1, 1, 3, 2, 2, 2], dtype=np.uint64)
    D = O.geodesics(masks, np.zeros(n, np.int32), [4], rp, col)
    # entries: one per body except body 3 (two)
    assert list(D[3:5]) == [1, 1]
    assert np.allclose(O.weights(D[3:5]), [0.5, 0.5])
    # two shared bodies {2,3}: D(2) = (1, 2), D(3) = (2, 1) -> (2/3, 1/3) and (1/3, 2/3)
    masks = np.array([1, 1, 3, 3, 2, 2, 2], dtype=np.uint64)
    D = O.geodesics(masks, np.zeros(n, np.int32), [4], rp, col)
    assert list(D[2:4]) == [1, 2] and list(D[4:6]) == [2, 1]
    assert np.allclose(O.weights(D[2:4]), [2 / 3, 1 / 3])
    assert np.allclose(O.weights(D[4:6]), [1 / 3, 2 / 3])
    # beta = 1 hides the far worker: weight 0 for it
    D = O.geodesics(masks, np.zeros(n, np.int32), [1], rp, col)
    assert list(D[2:4]) == [1, 255]
    assert np.allclose(O.weights(D[2:4]), [1.0, 0.0])


@pytest.mark.parametrize("seed", range(6))
def test_geodesics_match_floyd_warshall(seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import floyd_warshall
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 65))
    m = int(rng.integers(n, 3 * n))
    edges = rng.integers(0, n, size=(m, 2))
    edges = edges[edges[:, 0] != edges[:, 1]]
    rp, col = O.graph(n, np.ones(n), edges)
    n_workers = int(rng.integers(2, 5))
    masks = np.zeros(n, np.uint64)
    for b in range(n):
        k = 1 if rng.random() < 0.6 else int(rng.integers(2, n_workers + 1))
        ws = rng.choice(n_workers, size=k, replace=False)
        masks[b] = np.uint64(_bits(ws))
    beta = int(rng.integers(1, 5))
    D = O.geodesics(masks, np.zeros(n, np.int32), [beta], rp, col)
    A = csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    dist = floyd_warshall(A, unweighted=True)
    e = 0
    for o in range(n):
        ws = [w for w in range(64) if int(masks[o]) >> w & 1]
        for w in ws:
            if len(ws) >= 2:
                src = [b for b in range(n) if int(masks[b]) == 1 << w]
                d = min([dist[o, b] for b in src], default=np.inf)
                want = int(d) if d <= beta else 255
                assert D[e] == want, (o, w)
            else:
                assert D[e] == 255
            e += 1
    assert e == len(D)


def test_weights_are_convex():
    rng = np.random.default_rng(3)
    for _ in range(200):
        k = int(rng.integers(2, 9))
        D = rng.choice([1, 2, 3, 4, 5, 255], size=k).astype(np.uint8)
        w = O.weights(D)
        assert np.all(w >= 0) and abs(w.sum() - 1.0) < 1e-15
        finite = D != 255
        if finite.any():
            assert np.all(w[~finite] == 0)
            inv = 1.0 / D[finite]
            assert np.allclose(w[finite], inv / inv.sum())      # Eq 15 with D^-1
        else:
            assert np.allclose(w, 1.0 / k)


# ---------------------------------------------------------------------------
# Blend (Algorithm 4)
# ---------------------------------------------------------------------------

def _rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_blend_identical_copies_and_antipodes():
    rng = np.random.default_rng(1)
    for _ in range(20):
        s = rng.normal(size=13)
        s[3:7] = _rand_quat(rng)
        k = int(rng.integers(2, 6))
        copies = np.tile(s, (k, 1))
        w = rng.random(k)
        w /= w.sum()
        out = O.blend(copies, w)
        assert np.allclose(out, s, atol=1e-12)
        # the same rotation written as -q in some workers blends to +-q, never 0
        flip = rng.random(k) < 0.5
        flip[0] = False
        copies[flip, 3:7] *= -1
        out = O.blend(copies, w)
        assert np.allclose(out[3:7], s[3:7], atol=1e-12)
        assert abs(np.linalg.norm(out[3:7]) - 1) < 1e-14


def test_blend_weighted_means():
    rng = np.random.default_rng(2)
    q = _rand_quat(rng)
    copies = np.zeros((3, 13))
    for i in range(3):
        copies[i] = rng.normal(size=13)
        copies[i, 3:7] = q
    w = np.array([0.5, 0.3, 0.2])
    out = O.blend(copies, w)
    for sl in (slice(0, 3), slice(7, 10), slice(10, 13)):       # Eq 11-13
        assert np.allclose(out[sl], (w[:, None] * copies[:, sl]).sum(0), atol=1e-14)


# ---------------------------------------------------------------------------
# Colouring: greedy first-fit in priority order == networkx greedy_color
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_colouring_matches_networkx_greedy(seed):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(seed)
    n_local = int(rng.integers(5, 60))
    m = int(rng.integers(1, 150))
    slots = rng.integers(-1, n_local, size=(m, 2)).astype(np.int32)
    prio = np.array([O.mix64(int(x)) for x in rng.integers(0, 2**62, size=m)], dtype=np.uint64)
    ncol, colours = O.colour(slots, prio, n_local)
    Gr = nx.Graph()
    Gr.add_nodes_from(range(m))
    for u in range(m):
        for v in range(u + 1, m):
            su = {int(x) for x in slots[u] if x >= 0}
            sv = {int(x) for x in slots[v] if x >= 0}
            if su & sv:
                Gr.add_edge(u, v)
    order = sorted(range(m), key=lambda u: (-int(prio[u]), u))
    ref = nx.greedy_color(Gr, strategy=lambda g, c: iter(order))
    assert [ref[u] for u in range(m)] == list(colours)
    assert ncol == max(ref.values()) + 1


# ---------------------------------------------------------------------------
# Contacts: brute force and geometry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed", [(300, 0), (1200, 1), (2000, 2)])
def test_contacts_grid_equals_all_pairs(n, seed):
    sc = S.random_pile(n, seed, box=0.25 * n ** (1 / 3) + 1.0)
    st = sc.state.astype(np.float64)
    args = (st, sc.radius, sc.inv_mass, sc.planes)
    ab_g, phi_g, n_g, t_g = O.contacts(*args, use_grid=True)
    ab_b, phi_b, n_b, t_b = O.contacts(*args, use_grid=False)
    assert np.array_equal(ab_g, ab_b)
    assert np.array_equal(phi_g, phi_b)
    # independent FP64 geometry: pairs clearly inside / outside the margin
    p = st[:, :3]
    r = sc.radius.astype(np.float64)
    found = {(int(a), int(b)) for a, b in ab_g}
    d = np.linalg.norm(p[None, :, :] - p[:, None, :], axis=-1) - r[:, None] - r[None, :]
    iu = np.triu_indices(n, 1)
    for a, b, ph in zip(iu[0], iu[1], d[iu]):
        if ph < 0.05 - 1e-5:
            assert (a, b) in found
        elif ph > 0.05 + 1e-5:
            assert (a, b) not in found
    # canonical order and geometry of every record
    keys = ab_g[:, 0].astype(np.int64) * (1 << 32) + ab_g[:, 1]
    assert np.all(np.diff(keys) > 0)
    for (a, b), ph, nn, t1 in zip(ab_g, phi_g, n_g, t_g):
        if b < n:
            dv = p[b] - p[a]
            assert abs(ph - (np.linalg.norm(dv) - r[a] - r[b])) < 1e-12
            assert np.allclose(nn, dv / np.linalg.norm(dv), atol=1e-12)
        else:
            pl = sc.planes[b - n].astype(np.float64)
            assert abs(ph - (pl[:3] @ p[a] - pl[3] - r[a])) < 1e-12
            assert np.allclose(nn, -pl[:3])
        assert abs(np.linalg.norm(t1) - 1) < 1e-12 and abs(t1 @ nn) < 1e-12
        # built from the axis of the smallest |n_k|; a later axis wins only by
        # more than 1e-4 (the stated tie rule)
        an = np.abs(nn)
        k = 0
        if an[1] < an[0] - 1e-4:
            k = 1
        if an[2] < an[k] - 1e-4:
            k = 2
        assert abs(t1[k]) > 0.5


def test_pile_small_first_step_counts():
    # 8x8x4 lattice, spacing = diameter, jitter 0.01: 640 lattice neighbours
    # (224 + 224 + 192) and 64 ground contacts; 32 pairs straddle x = 0
    sc = S.pile_small()
    ab, phi, n, t1 = O.contacts(sc.state, sc.radius, sc.inv_mass, sc.planes)
    assert len(ab) == 704
    assert int(np.sum(ab[:, 1] == 256)) == 64
    sets = sc.set_of_body
    inter = [(a, b) for a, b in ab if b < 256 and sets[a] != sets[b]]
    assert len(inter) == 32


# ---------------------------------------------------------------------------
# PGS + integration: closed forms
# ---------------------------------------------------------------------------

def test_resting_sphere_takes_mgh():
    sc = S.resting_sphere(mass=2.0, dt=1.0 / 60.0)
    m, h = 1.0 / float(sc.inv_mass[0]), float(sc.scene_dt[0])   # the FP32 inputs
    sim = O.OracleSim(sc)
    x0 = sc.state.astype(np.float64)[0]
    sim.step()
    lam = sim.pairs()["lam"]
    assert lam.shape == (1, 3)
    assert abs(lam[0, 0] - m * G * h) < 1e-12 and np.all(lam[0, 1:] == 0)
    st = sim.state()[0]
    assert np.allclose(st[7:13], 0, atol=1e-15)
    assert np.allclose(st[:7], x0[:7], atol=1e-15)
    assert sim.metrics()["residual_rms"] < 1e-15
    # second step: warm start already holds m g h
    sim.step()
    assert abs(sim.pairs()["lam"][0, 0] - m * G * h) < 1e-12
    part, key, lam = sim.warmstart()
    assert list(part) == [0] and int(key[0]) == (0 << 32 | 1 << 2) and abs(lam[0, 0] - m * G * h) < 1e-12


def test_sphere_column_frictionless():
    k = 4
    sc = S.sphere_column(k=k, mass=1.0, dt=1.0 / 60.0, iters=400)
    m, h = 1.0 / float(sc.inv_mass[0]), float(sc.scene_dt[0])
    sim = O.OracleSim(sc)
    sim.step()
    ab, *_ = sim.contacts()
    lam = sim.pairs()["lam"]
    for (a, b), l in zip(ab, lam):
        if b == k:                                # ground carries the whole column
            want = k * m * G * h
        else:                                     # contact between a and a+1 carries k-1-a spheres
            want = (k - 1 - a) * m * G * h
        assert abs(l[0] - want) < 1e-9
    assert np.allclose(sim.state()[:, 7:13], 0, atol=1e-9)


@pytest.mark.parametrize("theta,mu", [(20.0, 0.5), (35.0, 0.9)])
def test_sphere_rolls_down_incline(theta, mu):
    sc = S.incline_sphere(theta_deg=theta, mass=1.5, radius=0.3, mu=mu, dt=1.0 / 60.0)
    m, r, h = 1.0 / float(sc.inv_mass[0]), float(sc.radius[0]), float(sc.scene_dt[0])
    assert mu >= 2.0 / 7.0 * math.tan(math.radians(theta))
    sim = O.OracleSim(sc)
    sim.step()
    th = math.radians(theta)
    npl = sc.planes[0, :3].astype(np.float64)
    th = math.atan2(-npl[0], npl[2])                             # the FP32 plane's angle
    st = sim.state()[0]
    v, w = st[7:10], st[10:13]
    # the FP32 plane normal is unit only to ~1e-8, hence relative 1e-7 bounds
    speed = 5.0 / 7.0 * G * math.sin(th) * h                    # a = 5/7 g sin(theta)
    assert abs(np.linalg.norm(v) - speed) < 1e-7 * speed
    assert abs(v @ npl) < 1e-7 * speed
    # rolling without slip: the contact point is at rest
    assert np.allclose(v + np.cross(w, -r * npl), 0, atol=1e-7 * speed)
    lam = sim.pairs()["lam"][0]
    assert abs(lam[0] - m * G * math.cos(th) * h) < 1e-7 * lam[0]
    ft = 2.0 / 7.0 * m * G * math.sin(th) * h
    assert abs(np.hypot(lam[1], lam[2]) - ft) < 1e-7 * ft


def test_sphere_slides_when_friction_too_small():
    theta = 30.0
    sc = S.incline_sphere(theta_deg=theta, mass=1.0, mu=0.1, dt=1.0 / 60.0)
    m, h, mu = 1.0 / float(sc.inv_mass[0]), float(sc.scene_dt[0]), float(sc.scene_mu[0])
    sim = O.OracleSim(sc)
    sim.step()
    npl = sc.planes[0, :3].astype(np.float64)
    th = math.atan2(-npl[0], npl[2])
    lam = sim.pairs()["lam"][0]
    assert abs(np.hypot(lam[1], lam[2]) - mu * lam[0]) < 1e-14   # on the friction bound
    v = sim.state()[0, 7:10]
    want = G * h * (math.sin(th) - mu * math.cos(th))
    assert abs(np.linalg.norm(v) - want) < 1e-7 * want


def test_pendulum_at_rest_and_swinging():
    sc0 = S.pendulum(mass=1.3, dt=1.0 / 120.0)
    m, h = 1.0 / float(sc0.inv_mass[0]), float(sc0.scene_dt[0])
    sim = O.OracleSim(sc0)
    sim.step()
    lam = sim.pairs()["lam"][0]
    assert np.allclose(lam, [0, 0, m * G * h], atol=1e-12)
    assert np.allclose(sim.state()[0, 7:13], 0, atol=1e-13)
    L = 1.0
    sc = S.pendulum(length=L, mass=1.3, angle_deg=40.0, dt=1.0 / 120.0)
    sim = O.OracleSim(sc)
    worst = 0.0
    heights = []
    for _ in range(600):
        sim.step()
        worst = max(worst, sim.metrics()["joint_gap_max"])
        heights.append(sim.state()[0, 2])
    assert worst < 1e-3 * L
    assert min(heights) < -0.99 * L                    # it swings through the bottom
    assert abs(np.linalg.norm(sim.state()[0, :3]) - L) < 1e-3 * L


def test_free_flight():
    sc = S.free_flight()
    h = float(sc.scene_dt[0])
    sim = O.OracleSim(sc)
    s0 = sc.state.astype(np.float64)
    sim.step()
    s1 = sim.state()
    g = np.array([0, 0, -G])
    assert np.allclose(s1[:, 7:10], s0[:, 7:10] + h * g, atol=1e-15, rtol=0)
    assert np.allclose(s1[:, 10:13], s0[:, 10:13], atol=0, rtol=0)
    assert np.allclose(s1[:, 0:3], s0[:, 0:3] + h * s1[:, 7:10], atol=1e-14)
    for i in range(s0.shape[0]):
        w = s0[i, 10:13]
        ang = np.linalg.norm(w) * h
        axis = w / np.linalg.norm(w)
        exact = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])   # q0 = identity
        assert np.allclose(s1[i, 3:7], exact, atol=ang ** 3)
        assert abs(np.linalg.norm(s1[i, 3:7]) - 1) < 1e-15


def _contact_rows_from_velocity_field(sc, ab, nrm, t1):
    """J rows built from the rigid-body velocity field at each contact point
    (independent of the oracle's lever-arm formulas)."""
    st = sc.state.astype(np.float64)
    n = sc.n_bodies
    rows = []
    for (a, b), nn, tt in zip(ab, nrm, t1):
        t2 = np.cross(nn, tt)
        xa, ra = st[a, :3], float(sc.radius[a])
        pc = xa + ra * nn                      # contact point on a's surface
        for d in (nn, tt, t2):
            J = np.zeros(6 * n)
            # w = d . (u_b(pc) - u_a(pc)), u(p) = v + w x (p - x)
            J[6 * a:6 * a + 3] = -d
            J[6 * a + 3:6 * a + 6] = -np.cross(pc - xa, d)
            if b < n:
                xb = st[b, :3]
                J[6 * b:6 * b + 3] = d
                J[6 * b + 3:6 * b + 6] = np.cross(pc - xb, d)
            rows.append(J)
    return np.array(rows)


def test_pgs_converges_to_enumerated_mlcp():
    """A spinning sphere driven into the corner of a floor and a wall: 6 rows.
    The converged PGS impulses must be the unique solution of the MLCP of
    Eq 5-7 found by enumerating every active set."""
    r, m, h, mu = 0.5, 1.25, 1.0 / 64.0, 0.375        # all exact in FP32
    th = math.radians(80.0)
    wall = [math.sin(th), 0.0, math.cos(th), 0.0]            # through the origin
    floor = [0.0, 0.0, 1.0, -2.0]
    # centre touching both planes exactly
    # n_w.c = r and z = r - 2  ->  c_x = (r - n_wz (r-2)) / n_wx
    cz = r - 2.0
    cx = (r - wall[2] * cz) / wall[0]
    sc = _scene([[cx, 0.3, cz]], [r], [1.0 / m], planes=[wall, floor], mu=mu, dt=h, iters=4000)
    st = sc.state.astype(np.float64)
    st[0, 7:10] = [-2.0, 0.7, -1.0]
    st[0, 10:13] = [3.0, -1.0, 2.0]
    sc.state = st.astype(np.float32)
    sim = O.OracleSim(sc)
    sim.step()
    ab, phi, nrm, t1 = sim.contacts()
    assert len(ab) == 2 and np.all(np.abs(phi) < 1e-6)
    lam_pgs = sim.pairs()["lam"].reshape(-1)
    st = sc.state.astype(np.float64)
    J = _contact_rows_from_velocity_field(sc, ab, nrm, t1)
    I = 0.4 * m * r * r
    Minv = np.diag([1 / m] * 3 + [1 / I] * 3)
    vstar = np.concatenate([st[0, 7:10] + h * np.array([0, 0, -G]), st[0, 10:13]])
    A = J @ Minv @ J.T
    w0 = J @ vstar
    target = np.array([(-p / h if p > 0 else 0.2 * max(-p - 0.001, 0) / h) if k == 0 else 0.0
                       for p in phi for k in range(3)])
    sols = []
    nrow = 6
    for states in itertools.product(*[("on", "off") if i % 3 == 0 else ("free", "hi", "lo")
                                      for i in range(nrow)]):
        # unknown lambda; equations per row state
        M = np.zeros((nrow, nrow))
        rhs = np.zeros(nrow)
        for i, s in enumerate(states):
            nrm_i = 3 * (i // 3)
            if s in ("on", "free"):
                M[i] = A[i]
                rhs[i] = target[i] - w0[i]
            elif s == "off":
                M[i, i] = 1.0
            elif s == "hi":
                M[i, i] = 1.0
                M[i, nrm_i] = -mu
            else:
                M[i, i] = 1.0
                M[i, nrm_i] = mu
        try:
            lam = np.linalg.solve(M, rhs)
        except np.linalg.LinAlgError:
            continue
        w = A @ lam + w0
        ok = True
        for i, s in enumerate(states):
            ln = lam[3 * (i // 3)]
            if s == "on":
                ok &= lam[i] >= -1e-12
            elif s == "off":
                ok &= w[i] >= target[i] - 1e-12
            elif s == "free":
                ok &= abs(lam[i]) <= mu * ln + 1e-12
            elif s == "hi":
                ok &= w[i] <= 1e-12
            else:
                ok &= w[i] >= -1e-12
        if ok:
            sols.append(lam)
    assert len(sols) >= 1
    for s in sols:
        assert np.allclose(s, sols[0], atol=1e-9)
    assert np.allclose(lam_pgs, sols[0], atol=1e-8)
    assert sim.metrics()["residual_rms"] < 1e-9


# ---------------------------------------------------------------------------
# whole-step invariants
# ---------------------------------------------------------------------------

def test_step_invariants_small_pile():
    sc = S.pile_small()
    sim = O.OracleSim(sc)
    for step in range(4):
        before = sim.state()
        sim.step()
        masks = sim.masks()
        assert all(_popc(x) >= 1 for x in masks)
        ent = sim.entries()
        ep, w, cp = ent["entry_ptr"], ent["weight"], ent["copies"]
        st = sim.state()
        for b in range(sc.n_bodies):
            k = ep[b + 1] - ep[b]
            assert k == _popc(masks[b])
            ww = w[ep[b]:ep[b + 1]]
            assert np.all(ww >= 0) and abs(ww.sum() - 1) < 1e-15
            if k == 1:                                   # a body in one set is not blended
                assert np.array_equal(st[b], cp[ep[b]])
            assert abs(np.linalg.norm(st[b, 3:7]) - 1) < 1e-14
        # no two constraints of one colour share a dynamic body in one worker
        pr = sim.pairs()
        ab, *_ = sim.contacts()
        seen = {}
        for p, kind, ci, c in zip(pr["part"], pr["kind"], pr["cidx"], pr["colour"]):
            assert kind == 0
            for body in ab[ci]:
                if body < sc.n_bodies:
                    key = (p, c, int(body))
                    assert key not in seen
                    seen[key] = 1
        assert not np.array_equal(before, st)


def test_single_worker_equals_unpartitioned_worker():
    # with one worker nothing is blended: every body takes its only copy
    sc = S.pile_small()
    sc.set_of_body[:] = 0
    sc.n_sets[:] = 1
    sim = O.OracleSim(sc)
    sim.step()
    assert sim.counts()["entries"] == sc.n_bodies
    assert np.array_equal(sim.entries()["copies"], sim.state())
