"""Box contact geometry on the GPU (one thread per pair) against the same
functions run on the host, bit for bit (both built without FMA
contraction; square roots and divisions are IEEE on both), on seeded
random batches at ragged sizes and at 60k pairs; the host runs are checked
against the FP64 oracle in tests/test_box_contacts.py."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import ovl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _q(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _boxes(rng, n):
    c = rng.normal(size=(n, 3))
    return np.concatenate([c, _q(rng, n)], axis=1).astype(np.float32), rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)


def _same(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("n", [0, 1, 127, 129, 60000])
def test_box_box_gpu_equals_host(n):
    rng = np.random.default_rng(31 + n)
    PA, HA = _boxes(rng, n)
    PB, HB = _boxes(rng, n)
    PB[:, :3] = PA[:, :3] + rng.normal(size=(n, 3)).astype(np.float32) * 0.8
    g = ovl.ovl_box_box_contacts(PA, HA, PB, HB, 0.05, on_gpu=True)
    h = ovl.ovl_box_box_contacts(PA, HA, PB, HB, 0.05, on_gpu=False)
    _same(g, h)
    if n == 60000:
        cnt, axis = g[0], g[4]
        assert np.sum(axis == -1) > 1000 and np.sum(axis >= 6) > 100 and np.sum(cnt == 4) > 1000


@pytest.mark.parametrize("n", [0, 1, 129, 60000])
def test_sphere_box_and_box_plane_gpu_equal_host(n):
    rng = np.random.default_rng(41 + n)
    P, H = _boxes(rng, n)
    S = np.concatenate([P[:, :3] + rng.normal(size=(n, 3)).astype(np.float32),
                        rng.uniform(0.1, 0.5, (n, 1)).astype(np.float32)], axis=1)
    _same(ovl.ovl_sphere_box_contacts(S, P, H, 0.05, on_gpu=True), ovl.ovl_sphere_box_contacts(S, P, H, 0.05, on_gpu=False))
    nn = rng.normal(size=(n, 3))
    nn /= np.maximum(np.linalg.norm(nn, axis=1, keepdims=True), 1e-12)
    PL = np.concatenate([nn, (np.sum(nn * P[:, :3], axis=1) - rng.uniform(-0.5, 1.5, n))[:, None]], axis=1).astype(np.float32)
    _same(ovl.ovl_box_plane_contacts(P, H, PL, 0.05, on_gpu=True), ovl.ovl_box_plane_contacts(P, H, PL, 0.05, on_gpu=False))


def test_stacked_boxes_on_gpu():
    # a 0.8 x 0.6 x 0.4 box resting 0.01 deep on a 2 x 2 x 1 box: four contacts at its bottom corners
    PA = np.array([[0, 0, 0, 1, 0, 0, 0]], np.float32)
    PB = np.array([[0.1, -0.2, 0.69, 1, 0, 0, 0]], np.float32)
    cnt, pts, gaps, nrm, axis = ovl.ovl_box_box_contacts(PA, [[1, 1, 0.5]], PB, [[0.4, 0.3, 0.2]], 0.02)
    assert cnt[0] == 4 and axis[0] in (2, 5)
    np.testing.assert_allclose(gaps[0], -0.01, atol=2e-6)
    np.testing.assert_allclose(nrm[0], [0, 0, 1], atol=1e-6)
    np.testing.assert_allclose(np.sort(pts[0, :, 0]), [-0.3, -0.3, 0.5, 0.5], atol=2e-6)

