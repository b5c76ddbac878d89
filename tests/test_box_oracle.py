"""Pins of the box-contact reference geometry (oracle/box_oracle.c), the
shapes of the paper's Building and Bridge scenes (Section 6), against facts
fixed independently of its formulas:

- closed forms: a box resting flat, tilted and corner-down on a plane; a
  sphere over a face, an edge, a corner and with its centre inside; small box
  on large and large on small (4-point manifolds, clipped corners); two
  crossed edges (one point, known gap), for each of the 9 edge axes;
- brute force: sphere-box distance against a dense sample of the box
  surface; box-box intersection against a linear-programming feasibility
  test (a point inside both boxes);
- the separating-axis theorem: over every sampled direction the separation
  never exceeds the best of the 15 candidate axes (overlapping boxes), and
  translating one box by the reported depth along the normal is exactly
  what separates them;
- invariance: a rigid motion of both shapes moves points and normals with it
  and leaves gaps unchanged."""
import numpy as np
import pytest

from oracle import box as X

ID = np.array([1.0, 0.0, 0.0, 0.0])


def qaxis(axis, ang):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * a])


def qmul(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_q(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def same_points(a, b, tol=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    if a.shape != b.shape:
        return False
    used = set()
    for p in a:
        d = np.linalg.norm(b - p, axis=1)
        j = int(np.argmin(d))
        if d[j] > tol or j in used:
            return False
        used.add(j)
    return True


FLOOR = [0.0, 0.0, 1.0, 0.0]


# ---- box on a plane --------------------------------------------------------
def test_box_plane_resting_flat_and_turned():
    h = [1.0, 0.5, 0.25]
    for ang in (0.0, 0.7):
        q = qaxis([0, 0, 1], ang)
        c = np.array([0.3, -0.2, 0.24])
        pts, gaps, n = X.box_plane(c, q, h, FLOOR, margin=0.02)
        assert pts.shape == (4, 3)
        np.testing.assert_allclose(gaps, -0.01, atol=1e-15)
        np.testing.assert_allclose(n, [0, 0, -1])
        R = rot(q)
        want = [c + R @ np.array([sx * 1.0, sy * 0.5, -0.25]) for sx in (-1, 1) for sy in (-1, 1)]
        assert same_points(pts, want, 1e-14)


def test_box_plane_tilted():
    h, th, cz = [1.0, 0.5, 0.25], 0.1, 0.4
    q = qaxis([1, 0, 0], th)
    pts, gaps, _ = X.box_plane([0, 0, cz], q, h, FLOOR, margin=1.0)
    # the bottom face's vertices: z = cz +- hy sin(th) - hz cos(th); two of each
    lo = cz - 0.5 * np.sin(th) - 0.25 * np.cos(th)
    hi = cz + 0.5 * np.sin(th) - 0.25 * np.cos(th)
    np.testing.assert_allclose(gaps, [lo, lo, hi, hi], atol=1e-15)
    # a margin between the two levels keeps only the lower edge
    pts, gaps, _ = X.box_plane([0, 0, cz], q, h, FLOOR, margin=0.5 * (lo + hi))
    assert gaps.shape == (2,) and np.allclose(gaps, lo)


def test_box_plane_corner_down_and_clear():
    a = 0.5
    # a cube with a body diagonal vertical: one lowest vertex at cz - a sqrt(3)
    q = qmul(qaxis([1, -1, 0], np.arccos(1 / np.sqrt(3))), ID)
    cz = a * np.sqrt(3) - 0.02
    pts, gaps, _ = X.box_plane([1.0, 2.0, cz], q, [a, a, a], FLOOR, margin=0.0)
    assert gaps.shape == (1,)
    np.testing.assert_allclose(gaps[0], -0.02, atol=1e-12)
    np.testing.assert_allclose(pts[0], [1.0, 2.0, -0.02], atol=1e-12)
    pts, gaps, _ = X.box_plane([0, 0, 5.0], ID, [a, a, a], FLOOR, margin=0.1)
    assert gaps.shape == (0,)


# ---- sphere on a box -------------------------------------------------------
H = np.array([1.0, 0.5, 0.25])


@pytest.mark.parametrize("s,pt,gap", [
    ((0.2, 0.1, 0.25 + 0.35), (0.2, 0.1, 0.25), 0.35 - 0.3),                      # over the top face
    ((1.1, 0.0, 0.35), (1.0, 0.0, 0.25), np.sqrt(0.02) - 0.3),                    # over an edge
    ((1.1, 0.6, 0.35), (1.0, 0.5, 0.25), np.sqrt(0.03) - 0.3),                    # over a corner
    ((0.9, 0.0, 0.0), (1.0, 0.0, 0.0), -0.1 - 0.3),                               # centre inside, +x face
    ((0.0, -0.45, 0.1), (0.0, -0.5, 0.1), -0.05 - 0.3),                           # inside, -y face
])
def test_sphere_box_closed_forms(s, pt, gap):
    hit, p, n, g = X.sphere_box(s, 0.3, [0, 0, 0], ID, H, margin=0.1)
    assert hit
    np.testing.assert_allclose(g, gap, atol=1e-15)
    np.testing.assert_allclose(p, pt, atol=1e-15)
    # the normal points from the sphere into the box: opposite the direction
    # from the surface point to the centre (outside), or the face normal
    np.testing.assert_allclose(np.linalg.norm(n), 1.0, atol=1e-15)
    if g + 0.3 > 0:
        d = np.array(s) - np.array(pt)
        np.testing.assert_allclose(n, -d / np.linalg.norm(d), atol=1e-14)


def _surface_samples(h, k=60):
    u = np.linspace(-1, 1, k)
    U, V = np.meshgrid(u, u)
    out = []
    for ax in range(3):
        o = [a for a in range(3) if a != ax]
        for sg in (-1, 1):
            P = np.zeros((k * k, 3))
            P[:, ax] = sg * h[ax]
            P[:, o[0]] = U.ravel() * h[o[0]]
            P[:, o[1]] = V.ravel() * h[o[1]]
            out.append(P)
    return np.concatenate(out)


def test_sphere_box_brute_force_distance_and_rigid_motion():
    rng = np.random.default_rng(3)
    surf = _surface_samples(H)
    step = 2 * H.max() / 59
    for _ in range(60):
        q, c = random_q(rng), rng.normal(size=3)
        R = rot(q)
        s = c + R @ (rng.uniform(-1, 1, 3) * (H + 0.6))
        hit, p, n, g = X.sphere_box(s, 0.2, c, q, H, margin=10.0)
        local = R.T @ (s - c)
        if np.all(np.abs(local) <= H):
            continue   # centre inside: the closed-form cases cover it
        world = c + surf @ R.T
        d_min = np.linalg.norm(world - s, axis=1).min()
        assert d_min - 0.2 >= g - 1e-12 and d_min - 0.2 <= g + step
        # a rigid motion of both: same gap, moved point and normal
        q2, t2 = random_q(rng), rng.normal(size=3)
        R2 = rot(q2)
        hit2, p2, n2, g2 = X.sphere_box(R2 @ s + t2, 0.2, R2 @ c + t2, qmul(q2, q), H, margin=10.0)
        np.testing.assert_allclose(g2, g, atol=1e-12)
        np.testing.assert_allclose(p2, R2 @ p + t2, atol=1e-12)
        np.testing.assert_allclose(n2, R2 @ n, atol=1e-12)


# ---- box on a box ----------------------------------------------------------
def test_box_box_small_on_large():
    hA, hB = [1.0, 1.0, 0.5], [0.4, 0.3, 0.2]
    for ang in (0.0, np.pi / 6):
        qB = qaxis([0, 0, 1], ang)
        cB = np.array([0.1, -0.2, 0.5 + 0.2 - 0.01])
        pts, gaps, n, axis, sep = X.box_box([0, 0, 0], ID, hA, cB, qB, hB, margin=0.02)
        assert axis == 2 and pts.shape == (4, 3)          # A's z face (ties go to A)
        np.testing.assert_allclose(n, [0, 0, 1], atol=1e-15)
        np.testing.assert_allclose(gaps, -0.01, atol=1e-14)
        np.testing.assert_allclose(sep, -0.01, atol=1e-14)
        R = rot(qB)
        want = [cB + R @ np.array([sx * 0.4, sy * 0.3, -0.2]) for sx in (-1, 1) for sy in (-1, 1)]
        assert same_points(pts, want, 1e-13)


def test_box_box_large_on_small_is_clipped():
    hA, hB = [0.4, 0.3, 0.2], [1.0, 1.0, 0.5]
    pts, gaps, n, axis, sep = X.box_box([0, 0, 0], ID, hA, [0.05, 0.0, 0.69], ID, hB, margin=0.02)
    assert axis == 2 and pts.shape == (4, 3)
    # the two z faces tie (-0.01 each): A's, the first scanned, is the reference.
    # B's bottom face (z = 0.19) clipped to A's top face, whose side planes are
    # moved out by the clipping tolerance (3e-4): A's top corners at z = 0.19
    tol = 3e-4
    want = [[sx * (0.4 + tol), sy * (0.3 + tol), 0.19] for sx in (-1, 1) for sy in (-1, 1)]
    assert same_points(pts, want, 1e-13)
    np.testing.assert_allclose(gaps, -0.01, atol=1e-14)


def test_box_box_crossed_edges():
    # A: a cube rotated 45 deg about x (its top is an edge along x at z = a sqrt 2);
    # B: a cube rotated 45 deg about y (its bottom is an edge along y), 0.01 lower than touching
    a = 0.5
    qA, qB = qaxis([1, 0, 0], np.pi / 4), qaxis([0, 1, 0], np.pi / 4)
    zB = 2 * a * np.sqrt(2) - 0.01
    pts, gaps, n, axis, sep = X.box_box([0, 0, 0], qA, [a, a, a], [0, 0, zB], qB, [a, a, a], margin=0.02)
    assert axis == 6 + 3 * 0 + 1                           # a_0 x b_1
    assert pts.shape == (1, 3)
    np.testing.assert_allclose(n, [0, 0, 1], atol=1e-14)
    np.testing.assert_allclose(gaps, [-0.01], atol=1e-13)
    np.testing.assert_allclose(pts[0], [0, 0, a * np.sqrt(2) - 0.005], atol=1e-13)
    # lifted past the margin: no contact
    pts, *_ = X.box_box([0, 0, 0], qA, [a, a, a], [0, 0, zB + 0.05], qB, [a, a, a], margin=0.02)
    assert pts.shape == (0, 3)


# rotations that bring a cube's local axis k onto world x (for A) or y (for B)
_TO_X = {0: ID, 1: qaxis([0, 0, 1], -np.pi / 2), 2: qaxis([0, 1, 0], np.pi / 2)}
_TO_Y = {1: ID, 0: qaxis([0, 0, 1], np.pi / 2), 2: qaxis([1, 0, 0], -np.pi / 2)}


@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("j", [0, 1, 2])
def test_box_box_every_edge_axis(i, j):
    """The crossed-edge pair with A's edge along its local axis i and B's
    along its local axis j (cubes, so relabelling the axes by a symmetry
    leaves the shapes alone): the chosen axis is a_i x b_j."""
    a = 0.5
    qA = qmul(qaxis([1, 0, 0], np.pi / 4), _TO_X[i])
    qB = qmul(qaxis([0, 1, 0], np.pi / 4), _TO_Y[j])
    zB = 2 * a * np.sqrt(2) - 0.01
    pts, gaps, n, axis, sep = X.box_box([0, 0, 0], qA, [a, a, a], [0, 0, zB], qB, [a, a, a], margin=0.02)
    assert axis == 6 + 3 * i + j
    np.testing.assert_allclose(n, [0, 0, 1], atol=1e-14)
    np.testing.assert_allclose(gaps, [-0.01], atol=1e-13)
    np.testing.assert_allclose(pts[0], [0, 0, a * np.sqrt(2) - 0.005], atol=1e-13)


def _lp_depth(cA, qA, hA, cB, qB, hB):
    """Largest t such that some point lies t inside both boxes (negative: the
    boxes would need growing by -t to meet) -- linear programming."""
    from scipy.optimize import linprog
    rows, rhs = [], []
    for c, q, h in ((cA, qA, hA), (cB, qB, hB)):
        R = rot(q)
        for k in range(3):
            e = R[:, k]
            rows.append(np.concatenate([e, [1.0]]))
            rhs.append(e @ c + h[k])
            rows.append(np.concatenate([-e, [1.0]]))
            rhs.append(-(e @ c) + h[k])
    res = linprog(c=[0, 0, 0, -1.0], A_ub=np.array(rows), b_ub=np.array(rhs),
                  bounds=[(None, None)] * 3 + [(None, 10.0)], method="highs")
    assert res.status == 0
    return -res.fun


def _configs(rng, n):
    for _ in range(n):
        hA, hB = rng.uniform(0.2, 1.0, 3), rng.uniform(0.2, 1.0, 3)
        qA, qB = random_q(rng), random_q(rng)
        cA = rng.normal(size=3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cB = cA + d * rng.uniform(0.2, 1.2) * (np.linalg.norm(hA) + np.linalg.norm(hB)) * 0.7
        yield cA, qA, hA, cB, qB, hB


def test_box_box_intersection_matches_linear_programming():
    rng = np.random.default_rng(5)
    seen = {True: 0, False: 0}
    for cA, qA, hA, cB, qB, hB in _configs(rng, 300):
        t = _lp_depth(cA, qA, hA, cB, qB, hB)
        if abs(t) < 1e-7:
            continue
        _, _, _, axis, _ = X.box_box(cA, qA, hA, cB, qB, hB, margin=0.0)
        separated = axis == -1
        assert separated == (t < 0)
        seen[separated] += 1
    assert seen[True] > 30 and seen[False] > 30


def _fibonacci(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def test_box_box_axes_attain_the_largest_separation():
    """For overlapping boxes the largest separation over all directions is
    attained on one of the 15 candidate axes (the separating-axis theorem)."""
    rng = np.random.default_rng(7)
    U = _fibonacci(40000)
    checked = 0
    for cA, qA, hA, cB, qB, hB in _configs(rng, 200):
        if _lp_depth(cA, qA, hA, cB, qB, hB) <= 1e-6:
            continue
        RA, RB = rot(qA), rot(qB)
        T = np.asarray(cB) - np.asarray(cA)
        sU = np.abs(U @ T) - np.abs(U @ RA) @ hA - np.abs(U @ RB) @ hB
        s15 = X.box_box_axes(cA, qA, hA, cB, qB, hB)
        assert sU.max() <= s15.max() + 1e-12
        assert sU.max() >= s15.max() - 0.05
        checked += 1
    assert checked > 40


def test_box_box_depth_is_the_separating_translation():
    rng = np.random.default_rng(9)
    checked = 0
    for cA, qA, hA, cB, qB, hB in _configs(rng, 200):
        pts, gaps, n, axis, sep = X.box_box(cA, qA, hA, cB, qB, hB, margin=0.0)
        if axis == -1 or sep > -1e-4:
            continue
        s15 = X.box_box_axes(cA, qA, hA, cB, qB, hB)
        # moving B along the normal by the depth (plus a little) separates them
        assert _lp_depth(cA, qA, hA, np.asarray(cB) + (-sep + 1e-6) * n, qB, hB) < 0
        if axis == int(np.argmax(s15)):
            # ... and a little less does not, when the chosen axis is the deepest one
            assert _lp_depth(cA, qA, hA, np.asarray(cB) + (-sep - 1e-6) * n, qB, hB) > 0
        # every contact is within the margin and the manifold has 1 to 4 points
        assert 1 <= pts.shape[0] <= 4 and np.all(gaps <= 0.0)
        checked += 1
    assert checked > 40


def test_box_box_rigid_motion_invariance():
    rng = np.random.default_rng(11)
    for cA, qA, hA, cB, qB, hB in _configs(rng, 80):
        out = X.box_box(cA, qA, hA, cB, qB, hB, margin=0.05)
        q2, t2 = random_q(rng), rng.normal(size=3)
        R2 = rot(q2)
        out2 = X.box_box(R2 @ cA + t2, qmul(q2, qA), hA, R2 @ cB + t2, qmul(q2, qB), hB, margin=0.05)
        assert out[3] == out2[3]
        if out[3] == -1:
            continue
        np.testing.assert_allclose(out2[4], out[4], atol=1e-12)
        np.testing.assert_allclose(out2[2], R2 @ out[2], atol=1e-12)
        np.testing.assert_allclose(out2[1], out[1], atol=1e-11)
        np.testing.assert_allclose(out2[0], out[0] @ R2.T + t2, atol=1e-11)


# ---- box rows: inertia and one box on a plane ------------------------------
def test_box_inertia_matches_a_dense_solid_grid():
    """R diag(1/I) R^T against the inverse of the inertia tensor summed over
    a 40^3 grid of the rotated solid (cell centres)."""
    rng = np.random.default_rng(13)
    k = 40
    u = (np.arange(k) + 0.5) / k * 2 - 1
    G = np.stack(np.meshgrid(u, u, u, indexing="ij"), axis=-1).reshape(-1, 3)
    for _ in range(4):
        h, q, m = rng.uniform(0.2, 1.5, 3), random_q(rng), rng.uniform(0.5, 5.0)
        P = (G * h) @ rot(q).T
        I = m / P.shape[0] * (np.sum(P * P) * np.eye(3) - P.T @ P)
        np.testing.assert_allclose(X.box_inv_inertia_world(q, h, 1.0 / m), np.linalg.inv(I),
                                   rtol=0, atol=2e-3 * np.abs(np.linalg.inv(I)).max())


M, G9, DT = 2.0, 9.81, 1.0 / 60.0


@pytest.mark.parametrize("yaw", [0.0, 0.7])
def test_box_resting_on_a_plane_carries_its_weight(yaw):
    h = [1.0, 0.5, 0.25]
    v, w, lam, pts, gaps = X.box_plane_step([0.3, -0.2, 0.25], qaxis([0, 0, 1], yaw), h, 1 / M, FLOOR,
                                            [0, 0, 0], [0, 0, 0], iters=500, dt=DT)
    assert lam.shape == (4, 3) and np.all(lam[:, 0] >= 0)
    np.testing.assert_allclose(lam[:, 0].sum(), M * G9 * DT, rtol=1e-12)
    np.testing.assert_allclose(v, 0, atol=1e-12)
    np.testing.assert_allclose(w, 0, atol=1e-12)


def test_box_sliding_decelerates_by_mu_g_dt_and_loads_its_front():
    """Sliding along x (t1 of a floor contact): Coulomb friction takes mu g dt
    off the speed; the friction's tipping moment about the centre is balanced
    by the normal impulses, so the front pair carries hz mu m g dt / hx more
    than the back pair, and the box does not turn."""
    hx, hy, hz, mu, v0 = 1.0, 0.5, 0.25, 0.5, 3.0
    v, w, lam, pts, gaps = X.box_plane_step([0, 0, hz], ID, [hx, hy, hz], 1 / M, FLOOR, [v0, 0, 0], [0, 0, 0],
                                            mu=mu, iters=3000, dt=DT)
    np.testing.assert_allclose(v, [v0 - mu * G9 * DT, 0, 0], atol=1e-10)
    np.testing.assert_allclose(w, 0, atol=1e-10)
    np.testing.assert_allclose(lam[:, 1].sum(), mu * lam[:, 0].sum(), rtol=1e-10)
    front = lam[pts[:, 0] > 0, 0].sum()
    back = lam[pts[:, 0] < 0, 0].sum()
    np.testing.assert_allclose(front - back, hz * mu * M * G9 * DT / hx, rtol=1e-8)


def test_box_push_out_of_a_penetration():
    """Every contact 0.01 deep: with erp 0.2 and no slop the normal rows aim
    at a separating speed of erp 0.01 / dt on top of cancelling gravity."""
    v, w, lam, pts, gaps = X.box_plane_step([0, 0, 0.25 - 0.01], ID, [1.0, 0.5, 0.25], 1 / M, FLOOR,
                                            [0, 0, 0], [0, 0, 0], erp=0.2, slop=0.0, iters=500, dt=DT)
    np.testing.assert_allclose(gaps, -0.01, atol=1e-15)
    np.testing.assert_allclose(v, [0, 0, 0.2 * 0.01 / DT], atol=1e-12)
    np.testing.assert_allclose(w, 0, atol=1e-12)
