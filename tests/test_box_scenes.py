"""The box workloads (stand-ins for the paper's Building and Two-way bridge
scenes, Section 6) are well formed, checked with the box reference geometry:
the building stands with every box supported and nothing interpenetrating;
the bridge's joints have coincident pivots and chain every plank to the
world at both ends.  The library's step does not take box bodies yet and
says so; the oracle's step does (tests/test_box_oracle_step.py)."""
import numpy as np
import pytest

from oracle import box as X
from oracle import oracle as O
from paper_2403_17261_gb300 import ovl
from paper_2403_17261_gb300 import scenes as S


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_building_stands_supported_without_overlap():
    sc = S.box_building(storeys=3, cells=4)
    he = sc.half_extents.astype(np.float64)
    box = np.nonzero(np.all(he > 0, axis=1))[0]
    sph = np.nonzero(np.all(he == 0, axis=1))[0]
    assert box.size == 3 * (25 + 16) and sph.size == 2
    st = sc.state.astype(np.float64)
    # the mass of a box is its volume (density 1)
    np.testing.assert_allclose(1.0 / sc.inv_mass[box], 8 * np.prod(he[box], axis=1), rtol=1e-6)
    # every box pair whose bounding spheres meet: no overlap deeper than 1e-6
    supported = np.zeros(sc.n_bodies, bool)
    for i in box:
        _, g, _ = X.box_plane(st[i, :3], st[i, 3:7], he[i], sc.planes[0].astype(np.float64), margin=1e-6)
        if g.size:
            assert g.min() >= -1e-6
            supported[i] = True
        for j in box:
            if j <= i or np.linalg.norm(st[i, :3] - st[j, :3]) > sc.radius[i] + sc.radius[j]:
                continue
            p, g, n, axis, sep = X.box_box(st[i, :3], st[i, 3:7], he[i], st[j, :3], st[j, 3:7], he[j], margin=1e-6)
            if g.size:
                assert sep >= -1e-6, (i, j, sep)
                # the upper box of a touching pair rests on the lower one
                up = j if st[j, 2] > st[i, 2] else i
                if abs(n[2]) > 0.99:
                    supported[up] = True
    assert np.all(supported[box])


def test_bridge_joints_chain_every_plank_to_the_world():
    sc = S.plank_bridge(planks=40)
    assert sc.joints.shape == (2 * 40 + 2, 2)
    st = sc.state.astype(np.float64)
    for (a, b), an in zip(sc.joints, sc.anchors.astype(np.float64)):
        pa = an[:3] if a < 0 else st[a, :3] + _rot(st[a, 3:7]) @ an[:3]
        pb = an[3:] if b < 0 else st[b, :3] + _rot(st[b, 3:7]) @ an[3:]
        np.testing.assert_allclose(pa, pb, atol=1e-6)
    # two joints at each end to the world, two between each pair of neighbours
    ends = np.sum(sc.joints < 0, axis=1)
    assert np.sum(ends) == 4
    inner = sc.joints[ends == 0]
    assert np.all(inner[:, 1] - inner[:, 0] == 1)
    assert np.bincount(inner[:, 0], minlength=39)[:39].min() == 2
    # default size: the paper's 3180 joints
    assert S.plank_bridge().joints.shape[0] == 3180


def test_box_scenes_upload_their_half_extents():
    sc = S.plank_bridge(planks=10)
    arr = ovl._SceneArrays(sc)
    assert arr.half is not None and np.array_equal(arr.half, sc.half_extents.astype(np.float32))
    assert bool(arr.desc.half_extents)
    # every box's radius bounds it (the step's broad phase tests bounding spheres)
    box = (sc.half_extents > 0).any(1)
    assert np.all(sc.radius[box] >= np.linalg.norm(sc.half_extents[box], axis=1) * (1 - 1e-6))
