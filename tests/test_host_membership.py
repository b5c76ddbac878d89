"""The library's host membership code (Algorithms 2-3 and 6-7, Section 5)
against the oracle, bit for bit, on seeded random scenes -- no GPU needed:
the C entry points ovl_host_load_balance / ovl_host_assign_overlap run the
same functions a step runs after reading its contacts back.

Scenes: spheres scattered in a box, contacts between centres closer than a
contact distance (canonical order: ascending (a, b)), workers as slabs along
x with half of the bodies near a slab boundary already in both neighbours
(as a previous step's activations leave them), several scenes per batch
with their own worker counts (2 to 64) and growth depths (0 to 3)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_17261_gb300 import ovl


def _scene(rng, n, n_sets, reach=0.9, overlap_band=0.6):
    side = (n / 1.5) ** (1 / 3)
    x = rng.uniform(0, side, size=(n, 3))
    from scipy.spatial import cKDTree
    pairs = np.array(sorted(cKDTree(x).query_pairs(reach)), dtype=np.int64).reshape(-1, 2)
    slab = np.minimum((x[:, 0] / side * n_sets).astype(np.int64), n_sets - 1)
    mask = (np.uint64(1) << slab.astype(np.uint64)).astype(np.uint64)
    # bodies near a slab boundary also belong to the neighbouring slab
    pos = x[:, 0] / side * n_sets - slab
    half = rng.random(n) < 0.5   # only some of them, so some contacts still cross
    lo = (pos < overlap_band / 2) & (slab > 0) & half
    hi = (pos > 1 - overlap_band / 2) & (slab < n_sets - 1) & half
    mask[lo] |= np.uint64(1) << (slab[lo] - 1).astype(np.uint64)
    mask[hi] |= np.uint64(1) << (slab[hi] + 1).astype(np.uint64)
    return pairs, mask


def _batch(seed, sizes, sets, gammas):
    rng = np.random.default_rng(seed)
    pairs, masks, sob = [], [], []
    base = 0
    for s, (n, k) in enumerate(zip(sizes, sets)):
        p, m = _scene(rng, n, k)
        pairs.append(p + base)
        masks.append(m)
        sob.append(np.full(n, s, np.int32))
        base += n
    n = base
    pairs = np.concatenate(pairs) if pairs else np.zeros((0, 2), np.int64)
    masks = np.concatenate(masks)
    sob = np.concatenate(sob)
    # CSR of the contact graph (sorted neighbour lists)
    adj = [[] for _ in range(n)]
    for a, b in pairs:
        adj[a].append(int(b))
        adj[b].append(int(a))
    row_ptr = np.zeros(n + 1, np.int32)
    row_ptr[1:] = np.cumsum([len(v) for v in adj])
    col = np.array([c for v in adj for c in sorted(v)], dtype=np.int32)
    count = np.bincount(pairs.ravel(), minlength=n).astype(np.int32)
    return dict(n=n, pairs=pairs, masks=masks, sob=sob, sets=np.array(sets, np.int32),
                gammas=np.array(gammas, np.int32), row_ptr=row_ptr, col=col, count=count)


BATCHES = [
    dict(seed=1, sizes=[600], sets=[4], gammas=[1]),
    dict(seed=2, sizes=[900], sets=[8], gammas=[2]),
    dict(seed=3, sizes=[400, 700, 250, 800], sets=[2, 5, 3, 16], gammas=[0, 1, 2, 3]),
    dict(seed=4, sizes=[1500], sets=[64], gammas=[2]),
]


@pytest.mark.parametrize("batch", BATCHES, ids=lambda b: f"seed{b['seed']}")
@pytest.mark.parametrize("act,deact", [(True, True), (True, False), (False, True)])
@pytest.mark.parametrize("weighted", [False, True])
def test_load_balance_matches_oracle(batch, act, deact, weighted):
    B = _batch(**batch)
    w = B["count"] if weighted else None
    want = O.load_balance(B["masks"], B["sob"], B["sets"], B["row_ptr"], B["col"], B["pairs"], B["gammas"],
                          do_activate=act, do_deactivate=deact,
                          weights=None if w is None else 1 + w.astype(np.int64))
    for threads in (1, 4):
        got = ovl.ovl_host_load_balance(B["masks"], B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"],
                                        B["pairs"], contact_count=w, do_activate=act, do_deactivate=deact,
                                        threads=threads)
        assert np.array_equal(got, want), (threads, int(np.sum(got != want)))
    # the pass moves something, so the comparison is not vacuous
    assert act is False or not np.array_equal(want, B["masks"]) or B["pairs"].shape[0] == 0


def test_load_balance_contact_order_matters():
    """Algorithm 6 is sequential: reversing the candidates changes the
    result on both sides in the same way."""
    B = _batch(seed=5, sizes=[800], sets=[6], gammas=[2])
    rev = B["pairs"][::-1].copy()
    want = O.load_balance(B["masks"], B["sob"], B["sets"], B["row_ptr"], B["col"], rev, B["gammas"])
    got = ovl.ovl_host_load_balance(B["masks"], B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"], rev)
    assert np.array_equal(got, want)
    fwd = ovl.ovl_host_load_balance(B["masks"], B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"],
                                    B["pairs"])
    assert not np.array_equal(fwd, got)


def test_load_balance_degenerate_inputs():
    B = _batch(seed=6, sizes=[300], sets=[3], gammas=[1])
    # no contacts: nothing changes
    got = ovl.ovl_host_load_balance(B["masks"], B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"],
                                    np.zeros((0, 2), np.int32))
    assert np.array_equal(got, B["masks"])
    # a mask bit outside the scene's workers is a membership error
    bad = B["masks"].copy()
    bad[0] |= np.uint64(1) << np.uint64(5)
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_host_load_balance(bad, B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"], B["pairs"])
    assert e.value.code == ovl.OVL_ERR_MEMBERSHIP
    # scenes out of order, or a contact across scenes, are argument errors
    sob2 = np.zeros(B["n"], np.int32)
    sob2[: B["n"] // 2] = 1   # scene 1's bodies before scene 0's
    with pytest.raises(ovl.OvlError):
        ovl.ovl_host_load_balance(B["masks"], sob2, [3, 3], [1, 1], B["row_ptr"], B["col"], B["pairs"])
    with pytest.raises(ovl.OvlError):
        ovl.ovl_host_load_balance(B["masks"], B["sob"], B["sets"], B["gammas"], B["row_ptr"], B["col"],
                                  np.array([[0, B["n"]]], np.int32))


def _joint_batch(seed, n, n_sets, n_joints, gamma):
    rng = np.random.default_rng(seed)
    # a random forest of joints over a line of bodies (neighbours in index
    # order are spatial neighbours), some static bodies and world joints
    set_of = np.minimum(np.arange(n) * n_sets // n, n_sets - 1)
    mask = (np.uint64(1) << set_of.astype(np.uint64)).astype(np.uint64)
    im = np.where(rng.random(n) < 0.05, 0.0, rng.uniform(0.5, 2.0, n)).astype(np.float32)
    mask[im == 0] = 0
    a = rng.integers(0, n, size=n_joints)
    b = np.clip(a + rng.integers(-4, 5, size=n_joints), -1, n - 1)
    b[rng.random(n_joints) < 0.05] = -1
    return dict(mask=mask, sob=np.zeros(n, np.int32), sets=np.array([n_sets], np.int32),
                gammas=np.array([gamma], np.int32), im=im, joints=np.stack([a, b], axis=1).astype(np.int32))


@pytest.mark.parametrize("seed,n,n_sets,n_joints,gamma", [(11, 400, 4, 500, 1), (12, 1000, 8, 1400, 2),
                                                          (13, 300, 3, 200, 0), (14, 2000, 16, 2600, 3)])
def test_assign_overlap_matches_oracle(seed, n, n_sets, n_joints, gamma):
    J = _joint_batch(seed, n, n_sets, n_joints, gamma)
    want = O.assign_overlap(J["mask"], J["sob"], J["sets"], J["im"].astype(np.float64), J["joints"], J["gammas"])
    got = ovl.ovl_host_assign_overlap(J["mask"], J["sob"], J["sets"], J["gammas"], J["im"], J["joints"])
    assert np.array_equal(got, want), int(np.sum(got != want))
    assert np.sum(got != J["mask"]) > 0
