"""Degenerate and boundary inputs, one oracle-checked step each: no contacts
at all, two spheres with coincident centres (the normal falls back to +z),
workers that hold no body, a static sphere carrying dynamic ones, zero PGS
sweeps (the warm start alone), and a timestep override."""
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


def _run(sc, warm=0, params=None, **step):
    P = _parity()
    orc, gpu = P.prepare(sc, warm_steps=warm, params=params)
    step.setdefault("stress", sc.name.startswith("random_pile"))
    try:
        return P.compare_step(orc, gpu, **step), gpu.stats()
    finally:
        gpu.close()


def test_no_contacts():
    rep, st = _run(S.free_flight(n=5))
    assert rep["contacts"] == 0 and st["n_pairs"] == 0 and st["device_status"] == 0


def test_coincident_centres():
    pos = np.array([(0.0, 0.0, 2.0), (0.0, 0.0, 2.0), (3.0, 0.0, 2.0)])
    sc = S._single("coincident", pos, np.full(3, 0.5), np.ones(3), [(0, 0, 1, 0)], mu=0.5, dt=1.0 / 60.0,
                   flags=1, gamma=0, beta=2, n_sets=2, set_of_body=[0, 1, 1])
    rep, st = _run(sc, params=dict(gravity=(0.0, 0.0, 0.0)))
    assert rep["contacts"] == 1
    from paper_2403_17261_gb300 import ovl
    g = ovl.Simulation(sc, dict(gravity=(0.0, 0.0, 0.0)))
    try:
        g.step()
        ab, phi, n, t1 = g.contacts()
        assert list(ab[0]) == [0, 1]
        np.testing.assert_array_equal(n[0], [0.0, 0.0, 1.0])
        assert phi[0] == -1.0
    finally:
        g.close()


def test_workers_without_bodies():
    # 300 spheres in 3 of 6 sets: workers 3-5 never receive a body
    sc = S.random_pile(300, 21, n_sets=6, box=0.3 * 300 ** (1 / 3) + 1.0)
    sc.set_of_body = (sc.set_of_body % 3).astype(np.int32)
    rep, st = _run(sc, warm=3)
    assert rep["contacts"] > 50
    assert st["n_workers"] == 6


def test_static_support():
    # a static sphere (inverse mass 0) under three dynamic ones in two workers
    pos = np.array([(0.0, 0.0, 0.5), (-0.5, 0.0, 1.4), (0.5, 0.0, 1.4), (0.0, 0.8, 1.4)])
    im = np.array([0.0, 1.0, 1.0, 1.0])
    sc = S._single("static_support", pos, np.full(4, 0.5), im, [(0, 0, 1, 0)], mu=0.5, dt=1.0 / 60.0,
                   flags=1, gamma=1, beta=4, n_sets=2, set_of_body=[0, 0, 1, 1])
    rep, st = _run(sc, warm=2)
    assert rep["contacts"] >= 5 and st["device_status"] == 0


def test_zero_sweeps_and_dt_override():
    sc = S.pile_small()
    rep, _ = _run(sc, warm=5, iters=0)
    assert rep["contacts"] > 600
    rep, _ = _run(sc, warm=5, dt=1.0 / 240.0)
    assert rep["contacts"] > 600
