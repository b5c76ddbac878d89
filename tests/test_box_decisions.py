"""Which box contacts exist, on which axis and at which clipped points are
integer decisions taken in FP32.  The oracle takes them itself in the
kernels' precision and operation order (oracle/box_oracle.c, *_f32), and
the library's functions (run on the host, which gives the GPU's bits) must
agree exactly on seeded random configurations: counts, axes, points, gaps
and normals equal."""
import numpy as np

from oracle import box as X
from paper_2403_17261_gb300 import ovl


def _q(rng, n):
    q = rng.normal(size=(n, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def test_box_box_decisions_match_exactly():
    rng = np.random.default_rng(71)
    n = 20000
    cA = rng.normal(size=(n, 3)).astype(np.float32)
    cB = (cA + rng.normal(size=(n, 3)) * 0.8).astype(np.float32)
    qA, qB = _q(rng, n), _q(rng, n)
    hA = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    hB = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    cnt, pts, gaps, nrm, axis = ovl.ovl_box_box_contacts(np.concatenate([cA, qA], 1), hA,
                                                         np.concatenate([cB, qB], 1), hB, 0.05, on_gpu=False)
    for i in range(n):
        p, g, nn, ax, _ = X.box_box_f32(cA[i], qA[i], hA[i], cB[i], qB[i], hB[i], margin=0.05)
        assert ax == axis[i] and p.shape[0] == cnt[i], i
        if ax == -1:
            continue
        assert np.array_equal(p, pts[i, : cnt[i]]) and np.array_equal(g, gaps[i, : cnt[i]]), i
        assert np.array_equal(nn, nrm[i]), i
    assert np.sum(axis == -1) > 1000 and np.sum(axis >= 6) > 100 and np.sum(cnt == 4) > 1000


def test_sphere_box_and_box_plane_decisions_match_exactly():
    rng = np.random.default_rng(72)
    n = 20000
    c = rng.normal(size=(n, 3)).astype(np.float32)
    q = _q(rng, n)
    h = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    s = np.concatenate([c + rng.normal(size=(n, 3)), rng.uniform(0.1, 0.5, (n, 1))], 1).astype(np.float32)
    cnt, pts, gaps, nrm = ovl.ovl_sphere_box_contacts(s, np.concatenate([c, q], 1), h, 0.05, on_gpu=False)
    for i in range(n):
        hit, p, nn, g = X.sphere_box_f32(s[i, :3], s[i, 3], c[i], q[i], h[i], margin=0.05)
        assert int(hit) == cnt[i] and g == gaps[i, 0] and np.array_equal(nn, nrm[i]), i
        if hit:
            assert np.array_equal(p, pts[i, 0]), i
    nn = rng.normal(size=(n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    pl = np.concatenate([nn, (np.sum(nn * c, 1) - rng.uniform(-0.5, 1.5, n))[:, None]], 1).astype(np.float32)
    cnt, pts, gaps, nrm = ovl.ovl_box_plane_contacts(np.concatenate([c, q], 1), h, pl, 0.05, on_gpu=False)
    for i in range(n):
        p, g, nv = X.box_plane_f32(c[i], q[i], h[i], pl[i], margin=0.05)
        assert p.shape[0] == cnt[i] and np.array_equal(p, pts[i, : cnt[i]]) and np.array_equal(g, gaps[i, : cnt[i]]), i
        assert np.array_equal(nv, nrm[i]), i
    assert np.sum(cnt == 4) > 1000 and np.sum(cnt == 0) > 1000
