"""Box bodies in the step (the Building and Bridge bodies of Section 6),
against the FP64 oracle from identical inputs, one step each: a building of
columns and slabs with balls dropped on it, a jointed plank bridge (ball
joints between box planks, the overlap grown over the joints by Algorithms
2-3), and a pit of mixed spheres and boxes.

Both sides decide box contacts in FP64 with the same stated tolerance rules,
so the contact lists (pairs, manifold index, order) must be equal -- also
for the pairs the oracle reports as near a threshold (counted and printed;
FP32 might decide those otherwise, FP64 computations in two orders agree far
closer) -- and the geometry equal to FP32 rounding.  Every other record as for spheres (tests/parity.py): graph,
masks after Algorithm 6, entries, D, pair order and colours bit for bit;
velocities at the stated 1e-4 m/s, positions at 1e-5 m."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _mixed(seed, n=300):
    """spheres and boxes dropped into a walled pit, some of them touching"""
    rng = np.random.default_rng(seed)
    side = (n / 2.0) ** (1 / 3) * 1.2
    pos = np.stack([rng.uniform(-side, side, n), rng.uniform(-side, side, n), rng.uniform(0.3, 2 * side, n)], 1)
    half = np.where(rng.random((n, 1)) < 0.5, rng.uniform(0.2, 0.6, (n, 3)), 0.0)
    rad = np.where(half[:, 0] > 0, np.linalg.norm(half, axis=1) * 1.0001, rng.uniform(0.2, 0.5, n))
    mass = np.where(half[:, 0] > 0, 8.0 * half.prod(axis=1), 4.0 / 3.0 * np.pi * rad ** 3)
    im = np.where(rng.random(n) < 0.1, 0.0, 1.0 / mass)
    planes = [[0, 0, 1, 0], [1, 0, 0, -side - 0.5], [-1, 0, 0, -side - 0.5]]
    sets = (pos[:, 0] > 0).astype(int) + 2 * (pos[:, 1] > 0).astype(int)
    sc = S._single("mixed_boxes", pos, rad, im, planes, mu=0.5, dt=1 / 60, flags=1, gamma=1, beta=4, n_sets=4,
                   set_of_body=sets)
    q = rng.normal(size=(n, 4))
    sc.state[:, 3:7] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    sc.half_extents = half.astype(np.float32)
    return sc


SCENES = {
    "building": (lambda: S.box_building(storeys=2, cells=3, balls=2, n_sets=4), [0, 5, 30]),
    "bridge": (lambda: S.plank_bridge(planks=40, balls=2, n_sets=3), [0, 5, 30]),
    "mixed": (lambda: _mixed(91), [0, 20, 40]),
}


@pytest.mark.parametrize("name,warm", [(k, w) for k, (_, ws) in SCENES.items() for w in ws])
def test_box_step_matches_oracle(name, warm):
    import parity as P
    sc = SCENES[name][0]()
    orc, gpu = P.prepare(sc, warm_steps=warm)
    try:
        rep = P.compare_step(orc, gpu)
        near = int(np.sum(orc.contact_ambiguity() < 1.0))
        k_o, p_o = orc.contact_points()
        k_g, p_g = gpu.contact_points()
        assert np.array_equal(k_o, k_g)
        np.testing.assert_allclose(p_g, p_o, atol=1e-5)
        he = sc.half_extents
        ab = orc.contacts()[0]
        n = sc.n_bodies
        boxy = (he[ab[:, 0]] > 0).any(1) | ((ab[:, 1] < n) & (he[np.minimum(ab[:, 1], n - 1)] > 0).any(1))
        assert boxy.sum() > 10
        print(f"\n  {name} after {warm} steps: {rep['contacts']} contacts ({int(boxy.sum())} with a box, {near} near a "
              f"decision threshold), |dv| {rep['v']:.2e} m/s, |dx| {rep['x']:.2e} m, |dlambda| {rep['lambda']:.2e}")
    finally:
        gpu.close()


def test_resting_box_on_gpu_carries_its_weight():
    """A box resting flat on the ground: four contacts whose normal impulses
    sum to m g h and no velocity left (closed form)."""
    from paper_2403_17261_gb300 import ovl
    m, h = 2.0, 1.0 / 60.0
    sc = S._single("box_rest", np.array([[0.3, -0.2, 0.25]]), np.array([np.sqrt(1.0 + 0.25 + 0.0625) * 1.0001]),
                   np.array([1.0 / m]), [[0, 0, 1, 0]], mu=0.5, dt=h, flags=1, gamma=0, beta=2, n_sets=1,
                   set_of_body=[0], iters=200)
    sc.half_extents = np.array([[1.0, 0.5, 0.25]], np.float32)
    g = ovl.Simulation(sc)
    try:
        g.step()
        lam = g.pairs()["lam"]
        assert lam.shape[0] == 4
        np.testing.assert_allclose(lam[:, 0].sum(), m * 9.81 * h, rtol=1e-5)
        assert np.abs(g.state()[0, 7:13]).max() < 1e-5
    finally:
        g.close()
