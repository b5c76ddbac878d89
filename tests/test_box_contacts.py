"""The library's FP32 box contact functions (box-plane, sphere-box, box-box;
the box bodies of the paper's Building and Bridge scenes, Section 6), run
on the host through the C ABI, against the FP64 reference geometry of
oracle/box_oracle.c on seeded random configurations.

Where FP32 may legitimately decide differently from FP64 the case is left
out: the oracle reports how close each pair's decisions came to their
thresholds (oracle/box_oracle.c), and pairs within one band of some
threshold are counted, not compared.  Everything else must agree: the
contact count, the chosen axis, and points, gaps and normals within 1e-6
(the library computes in FP64 and rounds its outputs to FP32 once)."""
import numpy as np
import pytest

from oracle import box as X
from paper_2403_17261_gb300 import ovl

# each comparison runs the library's functions on the host and, on a GPU
# machine, on the device (one thread per pair)
ON_GPU = [False, pytest.param(True, marks=pytest.mark.gpu, id="gpu")]


def _ensure_built(on_gpu):
    if on_gpu:
        import __graft_entry__ as g
        g.build()

TOL = 1e-6


def random_q(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def _match_sets(a, b, tol):
    """Greedy one-to-one matching of two point sets within tol."""
    if a.shape != b.shape:
        return False
    used = set()
    for p in a:
        d = np.linalg.norm(b - p, axis=1)
        d[list(used)] = np.inf
        j = int(np.argmin(d))
        if d[j] > tol:
            return False
        used.add(j)
    return True


def _pose(c, q):
    return np.concatenate([c, q]).astype(np.float32)


def _f64(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_box_box_host_matches_oracle(on_gpu):
    _ensure_built(on_gpu)
    rng = np.random.default_rng(21)
    n = 1500
    PA, HA, PB, HB = [], [], [], []
    for _ in range(n):
        hA, hB = rng.uniform(0.2, 1.0, 3), rng.uniform(0.2, 1.0, 3)
        cA = rng.normal(size=3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cB = cA + d * rng.uniform(0.2, 1.2) * (np.linalg.norm(hA) + np.linalg.norm(hB)) * 0.7
        PA.append(_pose(cA, random_q(rng)))
        PB.append(_pose(cB, random_q(rng)))
        HA.append(hA)
        HB.append(hB)
    PA, PB = np.array(PA), np.array(PB)
    HA, HB = np.array(HA, np.float32), np.array(HB, np.float32)
    margin = 0.05
    cnt, pts, gaps, nrm, axis = ovl.ovl_box_box_contacts(PA, HA, PB, HB, margin, on_gpu=on_gpu)
    compared = skipped = 0
    for i in range(n):
        # the oracle sees the same FP32 inputs, in FP64
        args = (_f64(PA[i, :3]), _f64(PA[i, 3:]), _f64(HA[i]), _f64(PB[i, :3]), _f64(PB[i, 3:]), _f64(HB[i]))
        p_o, g_o, n_o, ax_o, sep_o, amb = X.box_box(*args, margin=margin, with_amb=True)
        if amb < 1.0:
            skipped += 1
            continue
        assert axis[i] == ax_o, (i, axis[i], ax_o)
        assert cnt[i] == p_o.shape[0], (i, cnt[i], p_o.shape[0])
        if ax_o == -1:
            continue
        np.testing.assert_allclose(nrm[i], n_o, atol=TOL)
        k = cnt[i]
        assert _match_sets(pts[i, :k].astype(np.float64), p_o, TOL), i
        np.testing.assert_allclose(np.sort(gaps[i, :k]), np.sort(g_o), atol=TOL)
        compared += 1
    assert compared > 600 and skipped < n // 10
    # both decisions occur: separated pairs and contacts on faces and edges
    assert np.sum(axis == -1) > 100 and np.sum(axis >= 6) > 10 and np.sum((axis >= 0) & (axis < 6)) > 200


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_sphere_box_host_matches_oracle(on_gpu):
    _ensure_built(on_gpu)
    rng = np.random.default_rng(22)
    n = 2000
    S, P, H = [], [], []
    for _ in range(n):
        h = rng.uniform(0.2, 1.0, 3)
        q, c = random_q(rng), rng.normal(size=3)
        R = np.array(X_rot(q))
        s = c + R @ (rng.uniform(-1, 1, 3) * (h + 0.5))
        S.append(np.concatenate([s, [rng.uniform(0.1, 0.5)]]))
        P.append(_pose(c, q))
        H.append(h)
    S, P, H = np.array(S, np.float32), np.array(P), np.array(H, np.float32)
    margin = 0.05
    cnt, pts, gaps, nrm = ovl.ovl_sphere_box_contacts(S, P, H, margin, on_gpu=on_gpu)
    compared = 0
    for i in range(n):
        hit, p_o, n_o, g_o, amb = X.sphere_box(_f64(S[i, :3]), float(S[i, 3]), _f64(P[i, :3]), _f64(P[i, 3:]),
                                               _f64(H[i]), margin=margin, with_amb=True)
        if amb < 1.0:
            continue
        np.testing.assert_allclose(gaps[i, 0], g_o, atol=TOL)
        assert cnt[i] == int(hit), i
        np.testing.assert_allclose(nrm[i], n_o, atol=TOL)
        if hit:
            np.testing.assert_allclose(pts[i, 0], p_o, atol=TOL)
        compared += 1
    assert compared > 1800 and 300 < cnt.sum() < n


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_box_plane_host_matches_oracle(on_gpu):
    _ensure_built(on_gpu)
    rng = np.random.default_rng(23)
    n = 2000
    P, H, PL = [], [], []
    for _ in range(n):
        h = rng.uniform(0.2, 1.0, 3)
        nn = rng.normal(size=3)
        nn /= np.linalg.norm(nn)
        c = rng.normal(size=3)
        d = nn @ c - rng.uniform(-0.5, 1.5) * np.linalg.norm(h)
        P.append(_pose(c, random_q(rng)))
        H.append(h)
        PL.append(np.concatenate([nn, [d]]))
    P, H, PL = np.array(P), np.array(H, np.float32), np.array(PL, np.float32)
    margin = 0.05
    cnt, pts, gaps, nrm = ovl.ovl_box_plane_contacts(P, H, PL, margin, on_gpu=on_gpu)
    compared = 0
    for i in range(n):
        p_o, g_o, n_o, amb = X.box_plane(_f64(P[i, :3]), _f64(P[i, 3:]), _f64(H[i]), _f64(PL[i]), margin=margin,
                                         with_amb=True)
        if amb < 1.0:
            continue
        k = p_o.shape[0]
        assert cnt[i] == k, i
        np.testing.assert_allclose(nrm[i], n_o, atol=TOL)
        assert _match_sets(pts[i, :k].astype(np.float64), p_o, TOL), i
        np.testing.assert_allclose(np.sort(gaps[i, :k]), np.sort(g_o), atol=TOL)
        compared += 1
    assert compared > 1800 and np.sum(cnt == 4) > 100 and np.sum(cnt == 0) > 100


def X_rot(q):
    w, x, y, z = q
    return [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]


def test_box_contacts_reject_bad_arguments():
    rc = ovl.load_library().ovl_box_box_contacts(-1, None, None, None, None, 0.0, 0, None, None, None, None, None)
    assert rc == ovl.OVL_ERR_ARG
    rc = ovl.load_library().ovl_sphere_box_contacts(3, None, None, None, 0.0, 0, None, None, None, None)
    assert rc == ovl.OVL_ERR_ARG
    cnt, *_ = ovl.ovl_box_box_contacts(np.zeros((0, 7)), np.zeros((0, 3)), np.zeros((0, 7)), np.zeros((0, 3)), 0.0,
                                       on_gpu=False)
    assert cnt.shape == (0,)
