"""The library's FP32 box rows (general lever arms, full world inverse
inertia; the solve of Eq 1-7 for the box bodies of the paper's Section 6
scenes), run on the host through ovl_box_plane_step, against the FP64 oracle
(box_plane_step in oracle/box_oracle.c) on seeded random boxes resting on,
sinking into or lifting off random planes, and against the closed forms the
oracle is pinned to.  Velocities agree within the step's velocity tolerance
(1e-4 m/s + 1e-5 max|v|) after 50 sweeps, the solver's range; contact
counts exactly.

Over many more sweeps the two part: where every friction row of a box is
saturated (+-mu lambda_n), FP32 has no exact fixed point, the rows keep
exchanging impulse, and the rounding of those updates drifts the velocity
(1.4e-6 m/s per sweep on one such box, seed 61 item 424, while the FP64
iterate stands still from 300 to 10,000 sweeps)."""
import numpy as np

from oracle import box as X
from paper_2403_17261_gb300 import ovl

G, DT = 9.81, 1.0 / 60.0


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _qaxis(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * a])


def _qmul(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _batch(seed, n):
    """Half random orientations over random planes (1-2 contacts), half near
    flat on the floor (4 contacts), the deepest vertex within [-0.02, 0.015]
    of its plane."""
    rng = np.random.default_rng(seed)
    P, H, IM, PL, V = [], [], [], [], []
    for i in range(n):
        h = rng.uniform(0.2, 1.0, 3)
        c = rng.normal(size=3)
        if i % 2:
            q = rng.normal(size=4)
            q /= np.linalg.norm(q)
            nn = rng.normal(size=3)
            nn /= np.linalg.norm(nn)
        else:
            q = _qmul(_qaxis([0, 0, 1], rng.uniform(0, 6.3)), _qaxis(rng.normal(size=3), rng.uniform(0, 1e-3)))
            nn = np.array([0.0, 0.0, 1.0])
        R = _rot(q)
        lo = min(nn @ (c + R @ (np.array([sx, sy, sz]) * h)) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1))
        P.append(np.concatenate([c, q]))
        H.append(h)
        IM.append(rng.uniform(0.2, 2.0))
        PL.append(np.concatenate([nn, [lo - rng.uniform(-0.02, 0.015)]]))
        V.append(rng.normal(size=6) * 0.5)
    f = lambda x: np.array(x, np.float32)
    return f(P), f(H), f(IM), f(PL), f(V)


def _f64(x):
    return np.asarray(x, np.float32).astype(np.float64)


def test_box_rows_host_match_oracle():
    P, H, IM, PL, V = _batch(61, 600)
    vel, cnt, lam = ovl.ovl_box_plane_step(P, H, IM, PL, V, iters=50, on_gpu=False)
    for i in range(P.shape[0]):
        v, w, l, _, _ = X.box_plane_step(_f64(P[i, :3]), _f64(P[i, 3:]), _f64(H[i]), float(IM[i]), _f64(PL[i]),
                                         _f64(V[i, :3]), _f64(V[i, 3:]), iters=50, dt=DT)
        assert cnt[i] == l.shape[0], i
        ref = np.concatenate([v, w])
        np.testing.assert_allclose(vel[i], ref, atol=1e-4 + 1e-5 * np.abs(ref).max())
        np.testing.assert_allclose(lam[i, : cnt[i], 0].sum(), l[:, 0].sum(), atol=1e-4 / IM[i])
    assert np.sum(cnt == 4) > 200 and np.sum(cnt == 1) > 50


def test_box_rows_closed_forms():
    m, mu, v0, hx, hz = 2.0, 0.5, 3.0, 1.0, 0.25
    # resting: the normal impulses carry m g dt and nothing moves
    vel, cnt, lam = ovl.ovl_box_plane_step([[0.3, -0.2, hz, 1, 0, 0, 0]], [[hx, 0.5, hz]], [1 / m], [[0, 0, 1, 0]],
                                           [[0, 0, 0, 0, 0, 0]], mu=mu, iters=500, on_gpu=False)
    assert cnt[0] == 4
    np.testing.assert_allclose(lam[0, :, 0].sum(), m * G * DT, rtol=1e-5)
    np.testing.assert_allclose(vel[0], 0, atol=1e-5)
    # sliding along x: friction takes mu g dt off; the front pair carries
    # hz mu m g dt / hx more than the back pair; no turning
    vel, cnt, lam = ovl.ovl_box_plane_step([[0, 0, hz, 1, 0, 0, 0]], [[hx, 0.5, hz]], [1 / m], [[0, 0, 1, 0]],
                                           [[v0, 0, 0, 0, 0, 0]], mu=mu, iters=3000, on_gpu=False)
    np.testing.assert_allclose(vel[0], [v0 - mu * G * DT, 0, 0, 0, 0, 0], atol=1e-5)
    cnt_, pts, _, _ = ovl.ovl_box_plane_contacts([[0, 0, hz, 1, 0, 0, 0]], [[hx, 0.5, hz]], [[0, 0, 1, 0]], 0.02,
                                                 on_gpu=False)
    front = lam[0, pts[0, :, 0] > 0, 0].sum()
    back = lam[0, pts[0, :, 0] < 0, 0].sum()
    np.testing.assert_allclose(front - back, hz * mu * m * G * DT / hx, rtol=1e-4)
