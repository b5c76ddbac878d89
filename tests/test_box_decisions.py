"""Which box contacts exist, on which axis and at which clipped points are
decisions.  The library decides in FP32, the oracle in FP64, each with the
same stated tolerance rules (oracle/box_oracle.c header): a later axis or
face wins only by more than 0.3 mm (1e-4 in cosines), clipping keeps points
within 0.3 mm of a side plane, depth ties within 0.3 mm keep candidate
order.  The oracle reports how close each pair's decisions came to their
thresholds (in bands of 3e-5 m or 1e-5); pairs closer than one band are
ones FP32 may decide otherwise, and are counted, not compared.  Every other
pair must agree: count and axis exactly, points, gaps and normals within
1e-6 (in the same order): the library computes the geometry in FP64 too and
rounds its outputs to FP32 once.

Exactly aligned boxes -- stacks, columns on slabs, equal faces flush --
tie in exact arithmetic; under the rules they are never ambiguous."""
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


def _q(rng, n):
    q = rng.normal(size=(n, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def _f64(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _check_box_box(cA, qA, hA, cB, qB, hB, on_gpu):
    n = cA.shape[0]
    cnt, pts, gaps, nrm, axis = ovl.ovl_box_box_contacts(np.concatenate([cA, qA], 1), hA,
                                                         np.concatenate([cB, qB], 1), hB, 0.05, on_gpu=on_gpu)
    amb_n = 0
    for i in range(n):
        p, g, nn, ax, _, amb = X.box_box(_f64(cA[i]), _f64(qA[i]), _f64(hA[i]), _f64(cB[i]), _f64(qB[i]),
                                         _f64(hB[i]), margin=0.05, with_amb=True)
        if amb < 1.0:
            amb_n += 1
            continue
        if p.shape[0] == 0:
            assert cnt[i] == 0, i
            continue
        assert ax == axis[i] and p.shape[0] == cnt[i], (i, ax, axis[i], p.shape[0], cnt[i])
        np.testing.assert_allclose(pts[i, : cnt[i]], p, atol=TOL, err_msg=str(i))
        np.testing.assert_allclose(gaps[i, : cnt[i]], g, atol=TOL, err_msg=str(i))
        np.testing.assert_allclose(nrm[i], nn, atol=1e-6, err_msg=str(i))
    return cnt, axis, amb_n


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_box_box_decisions_agree(on_gpu):
    _ensure_built(on_gpu)
    rng = np.random.default_rng(71)
    n = 20000
    cA = rng.normal(size=(n, 3)).astype(np.float32)
    cB = (cA + rng.normal(size=(n, 3)) * 0.8).astype(np.float32)
    qA, qB = _q(rng, n), _q(rng, n)
    hA = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    hB = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    cnt, axis, amb_n = _check_box_box(cA, qA, hA, cB, qB, hB, on_gpu)
    assert amb_n <= 0.01 * n, amb_n
    assert np.sum(cnt == 0) > 1000 and np.sum(axis >= 6) > 100 and np.sum(cnt == 4) > 1000


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_aligned_boxes_are_never_ambiguous(on_gpu):
    _ensure_built(on_gpu)
    """Columns on slabs and stacked boxes: faces parallel, often flush, with
    exact ties between A's and B's faces and between clipped depths."""
    rng = np.random.default_rng(73)
    n = 3000
    right = np.array([[1, 0, 0, 0], [np.sqrt(0.5), 0, 0, np.sqrt(0.5)], [0, 0, 0, 1]], np.float64)
    qA = right[rng.integers(0, 3, n)].astype(np.float32)
    qB = right[rng.integers(0, 3, n)].astype(np.float32)
    # extents and offsets on a 0.1 m grid: side faces flush or 0.1 m apart,
    # never at the 0.05 m contact margin itself (that would be a real tie)
    hA = rng.choice([0.1, 0.2, 0.5, 1.0], size=(n, 3)).astype(np.float32)
    hB = np.where(rng.random((n, 1)) < 0.3, hA, rng.choice([0.1, 0.2, 0.5, 1.0], size=(n, 3))).astype(np.float32)
    cA = np.round(rng.uniform(-3, 3, (n, 3)), 1).astype(np.float32)
    # B on top of A (touching, or 1 cm in / 1 cm apart), slid along x, y by a multiple of 10 cm
    zh = []
    for i in range(n):
        ha = _f64(hA[i]) if qA[i, 0] == 1 or qA[i, 3] == 1 else _f64(hA[i])[[1, 0, 2]]
        hb = _f64(hB[i]) if qB[i, 0] == 1 or qB[i, 3] == 1 else _f64(hB[i])[[1, 0, 2]]
        zh.append(ha[2] + hb[2])
    off = np.stack([0.1 * rng.integers(-8, 9, n), 0.1 * rng.integers(-8, 9, n),
                    np.array(zh) + rng.choice([-0.01, 0.0, 0.01], n)], 1)
    cB = (cA + off).astype(np.float32)
    cnt, axis, amb_n = _check_box_box(cA, qA, hA, cB, qB, hB, on_gpu)
    assert amb_n == 0
    assert np.sum(cnt == 4) > 500


@pytest.mark.parametrize("on_gpu", ON_GPU)
def test_sphere_box_and_box_plane_decisions_agree(on_gpu):
    _ensure_built(on_gpu)
    rng = np.random.default_rng(72)
    n = 20000
    c = rng.normal(size=(n, 3)).astype(np.float32)
    q = _q(rng, n)
    h = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    s = np.concatenate([c + rng.normal(size=(n, 3)), rng.uniform(0.1, 0.5, (n, 1))], 1).astype(np.float32)
    cnt, pts, gaps, nrm = ovl.ovl_sphere_box_contacts(s, np.concatenate([c, q], 1), h, 0.05, on_gpu=on_gpu)
    amb_n = 0
    for i in range(n):
        hit, p, nn, g, amb = X.sphere_box(_f64(s[i, :3]), float(s[i, 3]), _f64(c[i]), _f64(q[i]), _f64(h[i]),
                                          margin=0.05, with_amb=True)
        if amb < 1.0:
            amb_n += 1
            continue
        assert int(hit) == cnt[i], i
        assert abs(gaps[i, 0] - g) <= TOL, i
        np.testing.assert_allclose(nrm[i], nn, atol=1e-6, err_msg=str(i))
        if hit:
            np.testing.assert_allclose(pts[i, 0], p, atol=TOL, err_msg=str(i))
    assert amb_n <= 0.01 * n, amb_n
    nn = rng.normal(size=(n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    pl = np.concatenate([nn, (np.sum(nn * c, 1) - rng.uniform(-0.5, 1.5, n))[:, None]], 1).astype(np.float32)
    cnt, pts, gaps, nrm = ovl.ovl_box_plane_contacts(np.concatenate([c, q], 1), h, pl, 0.05, on_gpu=on_gpu)
    amb_n = 0
    for i in range(n):
        p, g, nv, amb = X.box_plane(_f64(c[i]), _f64(q[i]), _f64(h[i]), _f64(pl[i]), margin=0.05, with_amb=True)
        if amb < 1.0:
            amb_n += 1
            continue
        assert p.shape[0] == cnt[i], i
        np.testing.assert_allclose(pts[i, : cnt[i]], p, atol=TOL, err_msg=str(i))
        np.testing.assert_allclose(gaps[i, : cnt[i]], g, atol=TOL, err_msg=str(i))
        np.testing.assert_allclose(nrm[i], nv, atol=1e-6, err_msg=str(i))
    assert amb_n <= 0.01 * n, amb_n
    assert np.sum(cnt == 4) > 1000 and np.sum(cnt == 0) > 1000
