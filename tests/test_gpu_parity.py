"""GPU parity: the CUDA path against the FP64 oracle, one step from identical
inputs, every record compared (see tests/parity.py for the tolerances)."""
import math

import numpy as np
import pytest

from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _parity():
    import parity
    return parity


@pytest.mark.parametrize("warm", [0, 1, 5, 20])
def test_pile_small(warm):
    P = _parity()
    orc, gpu = P.prepare(S.pile_small(), warm_steps=warm)
    rep = P.compare_step(orc, gpu)
    assert rep["contacts"] > 600


@pytest.mark.parametrize("cluster,limit", [(1, 0), (2, 0), (4, 0), (8, 0), (1, 16), (4, 16), (2, 40), (8, 20)])
def test_solver_paths(cluster, limit):
    """Every solver path: one CTA, clusters of 2 and 4 CTAs with the body state
    spread over their shared memory, and the global-memory path for workers
    above the shared-memory limit (also the colouring's scratch path)."""
    P = _parity()
    orc, gpu = P.prepare(S.pile_small(), warm_steps=3,
                         gpu_params=dict(pgs_cluster=cluster, smem_slot_limit=limit))
    P.compare_step(orc, gpu)


@pytest.mark.parametrize("warm", [0, 3])
def test_chain(warm):
    P = _parity()
    orc, gpu = P.prepare(S.chain(), warm_steps=warm)
    rep = P.compare_step(orc, gpu)
    assert rep["contacts"] > 2000


@pytest.mark.parametrize("n,seed,sets", [(300, 11, 3), (1500, 12, 5), (4000, 13, 8)])
def test_random_pile(n, seed, sets):
    P = _parity()
    sc = S.random_pile(n, seed, n_sets=sets, box=0.3 * n ** (1 / 3) + 1.0)
    orc, gpu = P.prepare(sc, warm_steps=2)
    P.compare_step(orc, gpu, stress=True)


@pytest.mark.parametrize("n_scenes,hi", [(12, 1024), (40, 300)])
def test_batched_scenes(n_scenes, hi):
    """Independent scenes of log-uniform sizes (piles and chains, 1-16 uneven
    sets each) stepped as one batch: every scene's records match the oracle."""
    P = _parity()
    sc = S.batched(seed=3, n_scenes=n_scenes, lo=64, hi=hi)
    orc, gpu = P.prepare(sc, warm_steps=2)
    rep = P.compare_step(orc, gpu)
    assert rep["contacts"] > 100


@pytest.mark.parametrize("warm", [45, 60, 70])
def test_contact_load_balance(warm):
    """Algorithm 6 with the contact load on a pile of big and small spheres
    (bodies with very unequal contact counts): the step's records match the
    oracle, membership bit for bit, and from the same inputs the body-count
    load decides differently (so the weights are what is being checked)."""
    from oracle import oracle as O
    P = _parity()
    sc = S.pile_mixed(seed=5, side=8, layers=8, n_sets=4)
    orc, gpu = P.prepare(sc, warm_steps=warm, params=dict(lb_load=1))
    try:
        by_count = O.OracleSim(sc, dict(lb_load=0))
        by_count.set_state(orc.state())
        by_count.set_masks(orc.masks())
        by_count.set_warmstart(*orc.warmstart())
        by_count.set_step_index(orc.step_index())
        rep = P.compare_step(orc, gpu)
        assert rep["contacts"] > 300
        by_count.step()
        assert not np.array_equal(by_count.masks(), gpu.membership())
    finally:
        gpu.close()


@pytest.mark.parametrize("weights", [0, 1])
def test_chain_weights_and_joint_error(weights):
    """The chain with Eq 15-16 weights or uniform ones: the step matches the
    oracle and uniform weights are exactly 1/|W_b|.  The joint violation the
    library measures matches the oracle's on the same FP32 state, before and
    after the step: the pivot differences of nearby coordinates are exact in
    FP32, so each gap is off by rotation and square-root rounding only
    (well below 1e-7 m for pivots 0.05 m from their centres)."""
    P = _parity()
    sc = S.chain()
    nj = sc.joints.shape[0]
    orc, gpu = P.prepare(sc, warm_steps=3, params=dict(weights=weights))
    try:
        def same_state_check():
            jo, jg = orc.joint_error(), gpu.joint_error()
            assert jo["sum"] > 1e-3
            assert abs(jg["sum"] - jo["sum"]) <= nj * 1e-7 and abs(jg["max"] - jo["max"]) <= 1e-7, (jo, jg)

        same_state_check()
        P.compare_step(orc, gpu)
        e = gpu.entries()
        k = np.diff(e["entry_ptr"])
        kk = np.repeat(k, k)
        shared = kk > 1
        assert shared.sum() > 20
        if weights == 1:
            np.testing.assert_array_equal(e["weight"][shared], (1.0 / kk[shared]).astype(np.float32))
        assert abs(orc.metrics()["joint_gap_sum"] - orc.joint_error()["sum"]) <= 1e-12
        orc.set_state(orc.state().astype(np.float32).astype(np.float64))
        gpu.set_state(orc.state().astype(np.float32))
        same_state_check()
    finally:
        gpu.close()


def test_contacts_beyond_the_register_list():
    """A sphere of radius 2 ringed by 60 spheres of radius 0.4 on its surface
    (golden-angle spiral): its neighbour list outgrows the 32 entries kept in
    registers and continues in its own global range; contacts, colours and
    the step still match the oracle."""
    P = _parity()
    k = 60
    i = np.arange(k) + 0.5
    z = 1.0 - 2.0 * i / k
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rr = np.sqrt(1.0 - z * z)
    u = np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)
    pos = np.concatenate([[[0.0, 0.0, 10.0]], [0.0, 0.0, 10.0] + 2.399 * u])
    rad = np.concatenate([[2.0], np.full(k, 0.4)])
    sc = S._single("ringed", pos, rad, np.ones(k + 1), [], mu=0.5, dt=1.0 / 60.0, flags=1, gamma=0,
                   beta=2, n_sets=1, set_of_body=np.zeros(k + 1, np.int32))
    orc, gpu = P.prepare(sc, params=dict(gravity=(0.0, 0.0, 0.0)))
    try:
        rep = P.compare_step(orc, gpu)
        ab = orc.contacts()[0]
        assert (ab[:, 0] == 0).sum() == k and rep["contacts"] >= k
    finally:
        gpu.close()


def test_closed_forms_on_gpu():
    from paper_2403_17261_gb300 import ovl
    sc = S.resting_sphere()
    g = ovl.Simulation(sc)
    g.step()
    lam = g.pairs()["lam"]
    m, h = 1.0 / float(sc.inv_mass[0]), float(sc.scene_dt[0])
    assert abs(lam[0, 0] - m * 9.81 * h) < 1e-6 * m * 9.81 * h
    assert np.abs(g.state()[0, 7:13]).max() < 1e-6


def test_launch_shapes_bit_identical():
    """Rows of one colour touch disjoint bodies, so every launch shape (CTAs
    per worker, threads, rows per thread) and the autotuner's pick compute
    the same bits."""
    from paper_2403_17261_gb300 import ovl
    sc = S.random_pile(3000, 21, n_sets=6, box=5.0)
    ref = None
    shapes = [dict(pgs_cluster=1, pgs_threads=512), dict(pgs_cluster=2, pgs_threads=256),
              dict(pgs_cluster=4, pgs_threads=512), dict(pgs_cluster=8, pgs_threads=256),
              dict(pgs_cluster=2, smem_slot_limit=64), dict(flags=ovl.OVL_FLAG_AUTOTUNE)]
    for kw in shapes:
        g = ovl.Simulation(sc, kw)
        for _ in range(3):
            g.step()
        st = g.state()
        if ref is None:
            ref = st
        else:
            assert np.array_equal(ref, st), kw
        if kw.get("flags"):
            txt = g.autotune_export()
            assert "cluster" in txt
            g2 = ovl.Simulation(sc, kw)
            g2.autotune_import(txt)
            assert g2.autotune_export() == txt
        g.close()
