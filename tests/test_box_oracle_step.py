"""Box bodies in the oracle's full step (row f1): contacts decided in FP32
(the box functions the library runs), one pair key per manifold point
(point index in bits 60-61; sphere keys unchanged), rows with lever arms to
the contact point and each box's world inverse inertia, then Algorithm 1
as for spheres.  Pinned to closed forms (a resting box, a sliding box, a
stack, a sphere on a box), to a building that stands in one worker and in
four with a growth depth that reaches every support, and to a bridge whose
joints hold in one worker and are all solved when it is partitioned."""
import numpy as np

from oracle import oracle as O
from paper_2403_17261_gb300 import scenes as S

G, DT = 9.81, 1.0 / 60.0
FLOOR = [[0.0, 0.0, 1.0, 0.0]]


def _scene(pos, half, inv_mass, radius=None, n_sets=1, set_of_body=None, iters=500, mu=0.5, vel=None):
    pos = np.asarray(pos, float)
    half = np.asarray(half, float)
    rad = np.linalg.norm(half, axis=1) if radius is None else np.asarray(radius, float)
    sc = S._single("boxes", pos, rad, inv_mass, FLOOR, mu=mu, dt=DT, flags=1, gamma=1, beta=4, n_sets=n_sets,
                   set_of_body=np.zeros(len(pos), int) if set_of_body is None else set_of_body, iters=iters)
    sc.half_extents = half.astype(np.float32)
    if vel is not None:
        sc.state[:, 7:13] = np.asarray(vel, np.float32)
    return sc


def test_resting_box_carries_its_weight_and_keys_its_points():
    m = 2.0
    sim = O.OracleSim(_scene([[0.3, -0.2, 0.25]], [[1.0, 0.5, 0.25]], [1 / m]))
    sim.step()
    st, pr = sim.state(), sim.pairs()
    np.testing.assert_allclose(st[0, 7:13], 0, atol=1e-9)
    np.testing.assert_allclose(pr["lam"][:, 0].sum(), m * G * DT, rtol=1e-6)
    keys = np.sort(pr["key"].astype(np.uint64))
    assert [int(k) & 3 for k in keys] == [0, 1, 2, 3]                     # the manifold's points
    assert all(int(k) >> 2 == 1 for k in keys)   # a = 0 (bits 32-57) against plane 0 (index n + 0 = 1)


def test_sliding_box_loses_mu_g_dt():
    m, mu, v0 = 2.0, 0.5, 3.0
    sim = O.OracleSim(_scene([[0.0, 0.0, 0.25]], [[1.0, 0.5, 0.25]], [1 / m], iters=3000, mu=mu,
                             vel=[[v0, 0, 0, 0, 0, 0]]))
    sim.step()
    np.testing.assert_allclose(sim.state()[0, 7:13], [v0 - mu * G * DT, 0, 0, 0, 0, 0], atol=1e-6)


def test_stack_of_two_boxes():
    # 2 kg under 1 kg; the floor carries both, the lower box the upper one
    m1, m2 = 2.0, 1.0
    sim = O.OracleSim(_scene([[0, 0, 0.25], [0.1, -0.05, 0.5 + 0.2]], [[1.0, 1.0, 0.25], [0.4, 0.3, 0.2]],
                             [1 / m1, 1 / m2], iters=2000))
    sim.step()
    st, pr = sim.state(), sim.pairs()
    np.testing.assert_allclose(st[:, 7:13], 0, atol=1e-7)
    key = pr["key"].astype(np.uint64)
    b = (key & np.uint64(0xFFFFFFFF)) >> np.uint64(2)
    ground = b == np.uint64(2)          # plane 0 is body index n + 0 = 2
    np.testing.assert_allclose(pr["lam"][ground, 0].sum(), (m1 + m2) * G * DT, rtol=1e-5)
    np.testing.assert_allclose(pr["lam"][~ground, 0].sum(), m2 * G * DT, rtol=1e-5)
    assert np.sum(~ground) == 4 and np.sum(ground) == 4


def test_sphere_resting_on_a_box():
    mb, ms, r = 2.0, 0.5, 0.3
    sim = O.OracleSim(_scene([[0, 0, 0.25], [0.2, 0.1, 0.5 + r]], [[1.0, 1.0, 0.25], [0, 0, 0]],
                             [1 / mb, 1 / ms], radius=[np.sqrt(2.0625), r], iters=2000))
    sim.step()
    st, pr = sim.state(), sim.pairs()
    np.testing.assert_allclose(st[:, 7:13], 0, atol=1e-7)
    b = (pr["key"].astype(np.uint64) & np.uint64(0xFFFFFFFF)) >> np.uint64(2)
    np.testing.assert_allclose(pr["lam"][b == np.uint64(1), 0].sum(), ms * G * DT, rtol=1e-5)
    np.testing.assert_allclose(pr["lam"][b == np.uint64(2), 0].sum(), (mb + ms) * G * DT, rtol=1e-5)


def _run(sc, steps):
    sim = O.OracleSim(sc)
    x0 = sim.state()[:, :3].copy()
    vmax = []
    for _ in range(steps):
        sim.step()
        vmax.append(np.abs(sim.state()[:, 7:10]).max())
    return sim, x0, np.array(vmax)


def test_building_stands_in_one_worker():
    sim, x0, vmax = _run(S.box_building(storeys=2, cells=2, balls=0, n_sets=1, iters=60), 15)
    assert vmax.max() < 1e-2
    assert np.abs(sim.state()[:, :3] - x0).max() < 5e-3


def test_partitioned_building():
    """With every supporting body inside each worker's reach (gamma 4) the
    partitioned building stands like the one-worker one.  (With gamma 0 a
    worker can hold a slab without all of its columns, and the slab drops
    for a step: about g h, the method's error at that depth.)"""
    sc = S.box_building(storeys=2, cells=2, balls=0, n_sets=4, iters=300)
    sc.scene_gamma[:] = 4
    sc.scene_beta[:] = 10
    sim, x0, vmax = _run(sc, 15)
    assert vmax.max() < 5e-3
    assert np.any([bin(int(m)).count("1") > 1 for m in sim.masks()])


def test_bridge_holds_in_one_worker():
    planks, height = 12, 4.0
    sim = O.OracleSim(S.plank_bridge(planks=planks, balls=0, n_sets=1, iters=300, height=height))
    worst = 0.0
    for _ in range(40):
        sim.step()
        worst = max(worst, sim.joint_error()["max"])
    z = sim.state()[:planks, 2]
    assert worst < 1e-2 and z.min() > height - 0.5 and z.min() < height - 1e-3


def test_partitioned_bridge_keeps_every_joint():
    """Two workers: the articulated assignment puts the joints across the
    boundary in the overlap, so every joint is solved by some worker, and the
    first steps match the one-worker accuracy.  (Over tens of steps the taut
    partitioned deck drifts further, as a taut chain of spheres does.)"""
    planks = 12
    sc = S.plank_bridge(planks=planks, balls=0, n_sets=2, gamma=2, beta=6, iters=300)
    sim = O.OracleSim(sc)
    sim.assign_overlap()
    for _ in range(5):
        sim.step()
    keys = sim.pairs()["key"].astype(np.uint64)
    joints = set(int(k) & ((1 << 62) - 1) for k in keys if int(k) >> 62 == 1)
    assert joints == set(range(sc.joints.shape[0]))
    assert sim.joint_error()["max"] < 2e-3


def test_sphere_on_a_static_box_platform():
    """A static box (inverse mass 0) as a platform: the sphere on it carries
    its weight, the box does not move and takes no rows of its own."""
    ms, r = 0.5, 0.3
    sim = O.OracleSim(_scene([[0, 0, 2.0], [0.2, 0.1, 2.25 + r]], [[1.0, 1.0, 0.25], [0, 0, 0]],
                             [0.0, 1 / ms], radius=[np.sqrt(2.0625), r], iters=500))
    x0 = sim.state()[0].copy()
    sim.step()
    st, pr = sim.state(), sim.pairs()
    np.testing.assert_array_equal(st[0], x0)
    np.testing.assert_allclose(st[1, 7:13], 0, atol=1e-9)
    assert len(pr["key"]) == 1
    np.testing.assert_allclose(pr["lam"][0, 0], ms * G * DT, rtol=1e-6)


def _incline(theta, mu):
    """a box resting flat on a plane tilted by theta about x"""
    h = np.array([0.5, 0.4, 0.2])
    n = np.array([0.0, -np.sin(theta), np.cos(theta)])
    c = n * h[2]                                        # bottom face on the plane through the origin
    sc = _scene([c], [h], [0.5], iters=2000, mu=mu)
    sc.planes = np.array([[n[0], n[1], n[2], 0.0]], np.float32)
    q = np.array([np.cos(theta / 2), np.sin(theta / 2), 0.0, 0.0])   # the box turned with the plane
    sc.state[0, 3:7] = q.astype(np.float32)
    return sc, n


def test_box_on_an_incline_sticks_below_the_friction_angle():
    sc, n = _incline(np.radians(20.0), mu=0.5)     # tan 20 = 0.36 < 0.5
    sim = O.OracleSim(sc)
    sim.step()
    # the FP32 contact points leave the four gaps ~1e-8 m uneven: a few 1e-6 of spin
    np.testing.assert_allclose(sim.state()[0, 7:13], 0, atol=1e-5)


def test_box_on_an_incline_slides_above_the_friction_angle():
    theta, mu = np.radians(35.0), 0.5               # tan 35 = 0.70 > 0.5
    sc, n = _incline(theta, mu)
    sim = O.OracleSim(sc)
    sim.step()
    v = sim.state()[0, 7:10]
    down = np.array([0.0, -np.cos(theta), -np.sin(theta)])   # down the slope
    np.testing.assert_allclose(v @ down, G * DT * (np.sin(theta) - mu * np.cos(theta)), rtol=1e-3)
    np.testing.assert_allclose(v @ n, 0, atol=1e-5)
    np.testing.assert_allclose(sim.state()[0, 10:13], 0, atol=1e-5)
