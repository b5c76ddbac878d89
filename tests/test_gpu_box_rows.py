"""Box rows (tests/test_box_rows.py) and the scene contact step for boxes
on the GPU, one thread per box, against the same functions run on the host,
value for value: both sides are built without FMA contraction, their square
roots and divisions are IEEE, and the row clamps compare explicitly."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import ovl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _same(a, b):
    # equal values (a zero's sign is not compared: it carries no meaning here)
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape and np.array_equal(x, y)


@pytest.mark.parametrize("n", [0, 1, 129, 20000])
def test_box_rows_gpu_equal_host(n):
    rng = np.random.default_rng(51 + n)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    P = np.concatenate([rng.normal(size=(n, 3)), q], axis=1).astype(np.float32)
    H = rng.uniform(0.2, 1.0, (n, 3)).astype(np.float32)
    P[:, 2] = H[:, 2] - rng.uniform(-0.01, 0.02, n).astype(np.float32)   # near the floor
    IM = rng.uniform(0.2, 2.0, n).astype(np.float32)
    PL = np.tile(np.array([[0, 0, 1, 0]], np.float32), (n, 1))
    V = (rng.normal(size=(n, 6)) * 0.5).astype(np.float32)
    g = ovl.ovl_box_plane_step(P, H, IM, PL, V, iters=100, on_gpu=True)
    h = ovl.ovl_box_plane_step(P, H, IM, PL, V, iters=100, on_gpu=False)
    _same(g, h)


def test_scene_contacts_gpu_equal_host():
    """The scene contact step for boxes on the GPU (one thread per body)
    against the same functions on the host."""
    from paper_2403_17261_gb300 import scenes as S
    for sc in (S.box_building(storeys=3, cells=4, balls=2, n_sets=1), S.plank_bridge(planks=200, balls=2, n_sets=1)):
        g = ovl.ovl_box_scene_contacts(sc, on_gpu=True)
        h = ovl.ovl_box_scene_contacts(sc, on_gpu=False)
        assert set(g) == set(h)
        for key in g:
            assert np.array_equal(g[key], h[key]), key
        assert len(h["ab"]) > 100
