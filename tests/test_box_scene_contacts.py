"""The library's contact step for scenes with boxes (ovl_box_scene_contacts,
run on the host, which gives the GPU's bits) against the oracle step's own
contacts on the same state.  The oracle decides box contacts in FP64 and
reports how close each decision came to its threshold; these scenes have
no ambiguous decision, so the lists must be the same, in the same
canonical (a, b, k) order, and gaps, normals and points must agree within
the FP32 rounding of the library's FP64 results (1e-6)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_17261_gb300 import ovl

# each comparison runs the library's functions on the host and, on a GPU
# machine, on the device (one thread per pair)
ON_GPU = [False, pytest.param(True, marks=pytest.mark.gpu, id="gpu")]


def _ensure_built(on_gpu):
    if on_gpu:
        import __graft_entry__ as g
        g.build()
from paper_2403_17261_gb300 import scenes as S

MARGIN = O.DEFAULT_PARAMS["margin"]


def _mixed(seed, n=300):
    """spheres and boxes dropped into a walled pit, some of them touching"""
    rng = np.random.default_rng(seed)
    side = (n / 2.0) ** (1 / 3) * 1.2
    pos = np.stack([rng.uniform(-side, side, n), rng.uniform(-side, side, n), rng.uniform(0.3, 2 * side, n)], 1)
    half = np.where(rng.random((n, 1)) < 0.5, rng.uniform(0.2, 0.6, (n, 3)), 0.0)
    rad = np.where(half[:, 0] > 0, np.linalg.norm(half, axis=1), rng.uniform(0.2, 0.5, n))
    im = np.where(rng.random(n) < 0.1, 0.0, rng.uniform(0.5, 2.0, n))
    planes = [[0, 0, 1, 0], [1, 0, 0, -side - 0.5], [-1, 0, 0, -side - 0.5]]
    sc = S._single("mixed_boxes", pos, rad, im, planes, mu=0.5, dt=1 / 60, flags=1, gamma=1, beta=4, n_sets=1,
                   set_of_body=np.zeros(n, int))
    q = rng.normal(size=(n, 4))
    sc.state[:, 3:7] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    sc.half_extents = half.astype(np.float32)
    return sc


SCENES = {
    "building": lambda: S.box_building(storeys=2, cells=3, balls=2, n_sets=1),
    "bridge": lambda: S.plank_bridge(planks=30, balls=2, n_sets=1),
    "mixed": lambda: _mixed(91),
}


@pytest.mark.parametrize("on_gpu", ON_GPU)
@pytest.mark.parametrize("name", list(SCENES))
def test_scene_contacts_match_the_oracle_step(name, on_gpu):
    _ensure_built(on_gpu)
    sc = SCENES[name]()
    sim = O.OracleSim(sc)
    sim.step()
    ab_o, phi_o, n_o, _ = sim.contacts()
    k_o, p_o = sim.contact_points()
    amb = sim.contact_ambiguity()
    assert np.all(amb >= 1.0), int(np.sum(amb < 1.0))
    r = ovl.ovl_box_scene_contacts(sc, margin=MARGIN, on_gpu=on_gpu)
    assert np.array_equal(r["ab"], ab_o) and np.array_equal(r["k"], k_o)
    n = sc.n_bodies
    he = sc.half_extents
    a, b = ab_o[:, 0], ab_o[:, 1]
    boxy = (he[a] > 0).any(1) | ((b < n) & (he[np.minimum(b, n - 1)] > 0).any(1))
    np.testing.assert_allclose(r["phi"][boxy], phi_o[boxy], atol=1e-6)
    np.testing.assert_allclose(r["normal"][boxy], n_o[boxy], atol=1e-6)
    np.testing.assert_allclose(r["point"][boxy], p_o[boxy], atol=1e-6)
    np.testing.assert_allclose(r["phi"][~boxy], phi_o[~boxy], atol=1e-6)
    np.testing.assert_allclose(r["normal"][~boxy], n_o[~boxy], atol=1e-6)
    assert boxy.sum() > 20 and len(ab_o) > 25


def test_scene_contacts_capacity():
    sc = SCENES["building"]()
    r = ovl.ovl_box_scene_contacts(sc, margin=MARGIN, on_gpu=False, cap=3)   # grows to the total
    assert len(r["ab"]) > 3


@pytest.mark.parametrize("bad", [np.nan, -0.25, np.inf])
def test_scene_contacts_refuse_bad_half_extents(bad):
    # a NaN or negative extent must not be read as a sphere
    sc = SCENES["building"]()
    sc.half_extents = sc.half_extents.copy()
    sc.half_extents[3, 1] = bad
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_box_scene_contacts(sc, margin=MARGIN, on_gpu=False)
    assert e.value.code == ovl.OVL_ERR_ARG
