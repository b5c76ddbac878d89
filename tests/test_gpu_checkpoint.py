"""Checkpoints (ovl_save / ovl_load) and ovl_step_n through the C ABI:
2N steps equal N steps, a save, a new context with the same scene, a load
and N more steps, bit for bit -- state, masks, warm-start cache and the step
index (which decides Algorithm 6's removal steps) all carried over."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _records(sim):
    part, key, lam = sim.warmstart()
    return [sim.state(), sim.membership(), part, key, lam]


@pytest.mark.parametrize("make,n", [(lambda: S.pile_small(), 6), (lambda: S.chain(), 3),
                                    (lambda: S.pile_large(side=16, n_sets=16), 75),
                                    (lambda: S.batched(n_scenes=12, hi=1024), 2)])
def test_save_load_resumes_bit_for_bit(make, n):
    from paper_2403_17261_gb300 import ovl
    sc = make()
    a = ovl.Simulation(sc)
    try:
        assert a.step_n(n) == n
        blob = a.save()
        assert ovl.checkpoint_step_index(blob) == n
        for _ in range(n):
            a.step()
        want = _records(a)
    finally:
        a.close()
    b = ovl.Simulation(sc)
    try:
        b.load(blob)
        assert b.step_index_value() == n
        b.step_n(n)
        got = _records(b)
    finally:
        b.close()
    for x, y in zip(want, got):
        assert x.dtype == y.dtype and x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))


def test_load_refuses_another_scene_and_bad_bytes():
    from paper_2403_17261_gb300 import ovl
    a = ovl.Simulation(S.pile_small())
    b = ovl.Simulation(S.random_pile(256, 3, n_sets=2))
    try:
        a.step()
        blob = a.save()
        with pytest.raises(ovl.OvlError) as e:
            b.load(blob)
        assert e.value.code == ovl.OVL_ERR_ARG
        with pytest.raises(ovl.OvlError):
            a.load(blob[:-1])
        with pytest.raises(ovl.OvlError):
            a.load(b"not a checkpoint" + blob[16:])
        a.load(blob)          # the intact checkpoint still loads
    finally:
        a.close()
        b.close()
