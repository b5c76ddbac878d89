"""ovl_geodesics_static (static scratch, no device allocation) against the
geodesic distances D(o,i) that ovl_step computes (Eq 16), called through the
C ABI twice in a row on the graphs of consecutive steps and then on another
scene, so that scratch left by one call must not leak into the next.

Collected last on purpose: it must also pass after every other test has used
the device."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _inputs(sim, torch):
    """The step's graph, masks and entries as device tensors, and a D buffer
    filled with a value every entry must overwrite."""
    row_ptr, col = sim.graph()
    mask = sim.membership()
    ent = sim.entries()
    dev = torch.device("cuda", 0)
    t = dict(
        rp=torch.from_numpy(row_ptr.astype(np.int32)).to(dev),
        col=torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).to(dev),
        mask=torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint64).view(np.int64)).to(dev),
        ep=torch.from_numpy(ent["entry_ptr"].astype(np.int32)).to(dev),
        D=torch.full((max(len(ent["D"]), 1),), 7, dtype=torch.uint8, device=dev),
        n_adj=len(col), ne=len(ent["D"]))
    return t, ent["D"], mask


def _call(sim, scene, t, torch):
    from paper_2403_17261_gb300 import ovl
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ovl.ovl_geodesics_static(sim.n, int(scene.n_sets[0]), int(scene.scene_beta[0]), t["rp"], t["col"],
                             t["n_adj"], t["mask"], t["ep"], t["ne"], t["D"], stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    return t["D"].cpu().numpy()[:t["ne"]]


def _static_D(sim, scene, torch):
    t, want, mask = _inputs(sim, torch)
    return _call(sim, scene, t, torch), want, mask


def test_static_geodesics_match_step_twice_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_2403_17261_gb300 import ovl
    sc = S.random_pile(1500, 12, n_sets=5, box=0.3 * 1500 ** (1 / 3) + 1.0)
    sim = ovl.Simulation(sc)
    try:
        for call in range(2):
            sim.step()
            got, want, mask = _static_D(sim, sc, torch)
            multi = np.array([bin(int(m)).count("1") for m in mask]) >= 2
            assert multi.any()                       # the overlap is not empty
            assert (want != 255).any()
            np.testing.assert_array_equal(got, want, err_msg=f"call {call}")
    finally:
        sim.close()


def test_static_geodesics_allocate_no_device_memory():
    """After one call (the module is loaded and the address looked up), a
    further call and its synchronize leave the device's free memory as it was."""
    torch = pytest.importorskip("torch")
    from paper_2403_17261_gb300 import ovl
    sc = S.random_pile(1500, 12, n_sets=5, box=0.3 * 1500 ** (1 / 3) + 1.0)
    sim = ovl.Simulation(sc)
    try:
        sim.step()
        t, want, _ = _inputs(sim, torch)
        np.testing.assert_array_equal(_call(sim, sc, t, torch), want)
        t["D"].fill_(7)
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        dev = torch.device("cuda", 0)
        ovl.ovl_geodesics_static(sim.n, int(sc.n_sets[0]), int(sc.scene_beta[0]), t["rp"], t["col"],
                               t["n_adj"], t["mask"], t["ep"], t["ne"], t["D"],
                               stream=torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after == free_before, (free_before, free_after)
        np.testing.assert_array_equal(t["D"].cpu().numpy()[:t["ne"]], want)
    finally:
        sim.close()


def test_static_geodesics_after_another_scene():
    torch = pytest.importorskip("torch")
    from paper_2403_17261_gb300 import ovl
    sc = S.chain()
    sim = ovl.Simulation(sc)
    try:
        sim.step()
        got, want, _ = _static_D(sim, sc, torch)
        assert (want != 255).any()
        np.testing.assert_array_equal(got, want)
    finally:
        sim.close()


def test_static_geodesics_rejects_sizes_beyond_the_limit():
    from paper_2403_17261_gb300 import ovl
    too_many = 4194304 // 64 + 1
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_geodesics_static(too_many, 64, 3, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.code == ovl.OVL_ERR_CAPACITY and "OVL_GEO_STATIC_MAX_PAIRS" in str(e.value)
    with pytest.raises(ovl.OvlError) as e:
        ovl.ovl_geodesics_static(10, 2, 255, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.code == ovl.OVL_ERR_CAPACITY and "OVL_GEO_STATIC_MAX_BETA" in str(e.value)
