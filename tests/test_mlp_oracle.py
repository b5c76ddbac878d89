"""Pins of the learned warm start's oracle: the FP64 network (oracle/mlp.py)
against finite differences, hand-worked values and Adam's closed forms, and
the contact features (oracle/ovl_oracle.c) against closed forms and brute
force on the constraint graph."""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_2403_17261_gb300 import scenes as S


def _rand(shape, seed):
    return np.asarray(S.SplitMix64(seed).uniform(int(np.prod(shape)), -1.0, 1.0)).reshape(shape)


def test_layout_matches_generator():
    assert M.N_PARAMS == S.MLP_N_PARAMS == 5187
    th = S.mlp_init_params(5)
    p = M.unpack(th)
    assert np.all(p["b1"] == 0) and np.all(p["b3"] == 0)
    assert np.abs(p["W1"]).max() <= np.sqrt(6 / 12) and np.abs(p["W2"]).max() <= np.sqrt(6 / 64)
    assert np.array_equal(M.pack(p), th.astype(np.float64))


def test_forward_hand_worked():
    # hidden units copy the inputs, output 0 sums their positive parts,
    # output 1 is minus that sum, output 2 is its bias; inputs 4-6 (the
    # previous impulses) are added to the three outputs
    p = {k: np.zeros(s) for k, s in M.SHAPES}
    p["W1"][np.arange(12), np.arange(12)] = 1.0
    p["W2"][np.arange(12), np.arange(12)] = 1.0
    p["W3"][:12, 0] = 1.0
    p["W3"][:12, 1] = -1.0
    p["b3"][:] = [0.5, 0.0, -2.0]
    x = np.array([[1.0, -2.0, 3.0, 0.0, 0.25, -0.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5]])
    y, _ = M.forward(M.pack(p), x)
    # 1 + 3 + 0.25 + 0.5 (+0.5 bias) + 0.25; -4.75 - 0.5; -2 + 0
    np.testing.assert_array_equal(y, [[5.5, -5.25, -2.0]])


def test_gradient_matches_central_differences():
    th = S.mlp_init_params(7).astype(np.float64) + 0.05 * _rand((M.N_PARAMS,), 8)
    X, T = S.synthetic_rows(9, seed=10)
    L, g = M.grad(th, X, T)
    assert abs(L - M.loss(th, X, T)) < 1e-15 * max(1.0, L)
    eps = 1e-6
    fd = np.empty_like(g)
    for i in range(M.N_PARAMS):
        e = np.zeros_like(th)
        e[i] = eps
        fd[i] = (M.loss(th + e, X, T) - M.loss(th - e, X, T)) / (2 * eps)
    # central differences are exact to O(eps^2) away from ReLU kinks
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-8 * np.abs(g).max())
    # every parameter block is exercised
    for name, sl in zip(("W1", "W2", "W3"), (slice(0, 768), slice(832, 4928), slice(4992, 5184))):
        assert np.abs(g[sl]).max() > 0, name


def test_zero_layers_give_the_previous_impulses():
    th = np.zeros(M.N_PARAMS)
    X, _ = S.synthetic_rows(50, seed=13)
    y, _ = M.forward(th, X)
    np.testing.assert_array_equal(y, X[:, 4:7].astype(np.float64))


def test_zero_loss_at_exact_targets():
    th = S.mlp_init_params(11).astype(np.float64)
    X, _ = S.synthetic_rows(20, seed=12)
    Y, _ = M.forward(th, X)
    L, g = M.grad(th, X, Y)
    assert L == 0.0 and np.all(g == 0.0)


def test_adam_first_step_is_a_sign_step():
    # with m and v started at zero, bias correction gives mhat = g and
    # vhat = g^2 on the first step, so the step is lr * g / (|g| + eps)
    th = np.zeros(5)
    g = np.array([3.0, -0.5, 1e-3, -7.0, 0.0])
    th1, m, v = M.adam(th, np.zeros(5), np.zeros(5), g, 1, lr=1e-3)
    np.testing.assert_allclose(th1, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_constant_gradient_keeps_its_step():
    # a constant gradient keeps mhat = g and vhat = g^2 for every t
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    g = np.array([2.0, -1.0, 0.25])
    for t in range(1, 40):
        prev = th
        th, m, v = M.adam(th, m, v, g, t, lr=0.01)
        np.testing.assert_allclose(th - prev, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_warm_start_projection():
    p = {k: np.zeros(s) for k, s in M.SHAPES}
    p["b3"][:] = [-1.0, 0.7, -0.2]
    lam = M.warm_start(M.pack(p), np.zeros((2, 12)), [2.0, 3.0], [0.5, 0.5])
    np.testing.assert_array_equal(lam, np.zeros((2, 3)))   # negative normal -> 0, friction -> 0
    p["b3"][:] = [1.0, 0.7, -0.2]
    lam = M.warm_start(M.pack(p), np.zeros((1, 12)), [2.0], [0.5])
    np.testing.assert_allclose(lam, [[2.0, 1.0, -0.4]])      # friction clamped to mu * 2


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------

def test_features_resting_sphere():
    sc = S.resting_sphere(mass=2.0)
    o = O.OracleSim(sc)
    o.step()
    f1 = o.features()
    assert not f1["found"][0] and np.all(f1["feat"][0, 4:7] == 0)
    o.step()
    f = o.features()
    h, m = float(sc.scene_dt[0]), 1.0 / float(sc.inv_mass[0])
    assert f["found"][0]
    # lambda_n = m g h exactly at phi = 0 (the resting-sphere closed form), and
    # s = g h m, so the scaled previous impulse is 1
    np.testing.assert_allclose(f["scale"][0], 9.81 * h * m, rtol=1e-15)
    np.testing.assert_allclose(f["feat"][0], [0, 0, 0, 0, 1, 0, 0, 1 / m, 0, 0, 0, 1.0],
                               atol=1e-12)


def test_features_spinning_sphere_on_plane():
    # contact point velocity of a sphere spinning about y at w: (w r, 0, 0)
    # relative to the plane; n = -z, t1 = x, t2 = n x t1 = -y
    sc = S.spinning_sphere(omega_y=3.0, height=0.49, radius=0.5)
    o = O.OracleSim(sc)
    o.step()
    f = o.features()["feat"][0]
    g, h = 9.81, float(sc.scene_dt[0])
    np.testing.assert_allclose(f[0:3], [0.0, 3.0 * 0.5 / (g * h), 0.0], atol=1e-12)
    np.testing.assert_allclose(f[3], (0.5 - np.float32(0.49)) / (g * h * h), rtol=1e-6)


def test_features_head_on_pair():
    sc = S.head_on(speed=1.0)
    o = O.OracleSim(sc, dict(gravity=(0.0, 0.0, 0.0)))
    o.step()
    F = o.features()
    h = float(sc.scene_dt[0])
    # g_ref = 1 without gravity; n = +x, closing speed 2; t1 = y, t2 = z
    np.testing.assert_allclose(F["feat"][0], [-2.0 / h, 0, 0, 0, 0, 0, 0, 1, 1, 1 / 8, 1 / 8, 1.0],
                               atol=1e-12)
    np.testing.assert_allclose(F["scale"][0], h / 2, rtol=1e-15)


def _graph_from_contacts(o, sc):
    nx = pytest.importorskip("networkx")
    ab = o.contacts()[0]
    n = sc.n_bodies
    G = nx.Graph()
    G.add_nodes_from(int(b) for b in range(n) if sc.inv_mass[b] > 0)
    for a, b in ab:
        if b < n and sc.inv_mass[a] > 0 and sc.inv_mass[b] > 0:
            G.add_edge(int(a), int(b))
    for a, b in sc.joints:
        if a >= 0 and b >= 0 and sc.inv_mass[a] > 0 and sc.inv_mass[b] > 0:
            G.add_edge(int(a), int(b))
    return nx, G


@pytest.mark.parametrize("make", [lambda: S.pile_small(), lambda: S.random_pile(400, 21, n_sets=4, box=2.5)])
def test_features_degree_and_depth_brute_force(make):
    sc = make()
    o = O.OracleSim(sc)
    o.step()
    o.step()
    F, P = o.features(), o.pairs()
    nx, G = _graph_from_contacts(o, sc)
    mask = o.masks()
    O_set = [b for b in G.nodes if bin(int(mask[b])).count("1") >= 2]
    assert O_set
    dist = nx.multi_source_dijkstra_path_length(G, O_set)
    depth = {b: min(dist.get(b, 8), 8) for b in G.nodes}
    ab = o.contacts()[0]
    n = sc.n_bodies
    checked = 0
    for q in range(len(P["kind"])):
        if P["kind"][q] != 0:
            continue
        a, b = ab[P["cidx"][q]]
        ends = [x for x in (a, b) if x < n and sc.inv_mass[x] > 0]
        deg = [G.degree(int(x)) / 8 if (x < n and sc.inv_mass[x] > 0) else 0.0 for x in (a, b)]
        assert F["feat"][q, 9] == deg[0] and F["feat"][q, 10] == deg[1]
        assert F["feat"][q, 11] == min(depth[int(x)] for x in ends) / 8
        checked += 1
    assert checked > 100
    assert np.array_equal(F["depth"][list(G.nodes)], [depth[b] for b in G.nodes])
