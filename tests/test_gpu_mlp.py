"""GPU parity of the learned warm start: contact features against the FP64
oracle from identical inputs, the tensor-core forward pass and the training
kernels' gradients against the FP64 network (tolerances from tests/mlp_bounds.py),
Adam's first step, the warm-start modes inside a step, and the solve log."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu

G = 9.81


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _parity():
    import parity
    return parity


def _bounds():
    import mlp_bounds
    return mlp_bounds


def _feature_tolerance(F, scale, h, terms=None):
    """Per-feature tolerance from the step's contact-geometry tolerance
    (normals, tangents and gaps within 1e-5 of the oracle) and FP32 rounding
    of identical inputs; integer-valued features are exact.  terms (per
    pair): |v_A| + |v_B| + r_A |w_A| + r_B |w_B| / (g h), the size of the
    velocity terms whose FP32 sum J v is (a rolling contact cancels them to
    ~0); J v is held to ~5 FP32 roundings of that size on top."""
    P = _parity()
    F = np.asarray(F, dtype=np.float64)
    tol = np.zeros_like(F)
    speed = np.linalg.norm(F[:, 0:3], axis=1, keepdims=True)
    tol[:, 0:3] = 2 * P.TOL_GEOM * speed + 1e-5 * np.abs(F[:, 0:3]) + 1e-6
    if terms is not None:
        tol[:, 0:3] += 3e-7 * np.asarray(terms, dtype=np.float64)[:, None]
    tol[:, 3] = P.TOL_GEOM / (G * h * h) + 1e-6 * np.abs(F[:, 3])
    tol[:, 4:7] = 2e-6 * np.abs(F[:, 4:7]) + 1e-7
    return tol


@pytest.mark.parametrize("make,warm", [(lambda: S.pile_small(), 5), (lambda: S.chain(), 2),
                                       (lambda: S.random_pile(1500, 12, n_sets=5, box=0.3 * 1500 ** (1 / 3) + 1.0), 2)])
def test_features_match_oracle(make, warm):
    from paper_2403_17261_gb300 import ovl
    P = _parity()
    sc = make()
    orc, gpu = P.prepare(sc, warm_steps=warm, gpu_params=dict(flags=ovl.OVL_FLAG_FEATURES))
    try:
        st0 = orc.state()
        P.compare_step(orc, gpu, stress=sc.name.startswith("random_pile"))
        Fo, Fg = orc.features(), gpu.features()
        assert np.array_equal(Fo["found"], Fg["found"])
        kind = orc.pairs()["kind"]
        assert (kind == 0).sum() > 100 and Fo["found"].any()
        h = float(sc.scene_dt[0])
        # size of the velocity terms of every pair's J v (static ends and planes: 0)
        keys = orc.pairs()["key"]
        joint = (keys >> np.uint64(62)) & np.uint64(1)
        a_i = (keys >> np.uint64(32)).astype(np.int64) & 0x3FFFFFF
        b_i = ((keys & np.uint64(0xFFFFFFFF)) >> np.uint64(2)).astype(np.int64)
        def mag(x):
            ok = (x < sc.n_bodies) & (joint == 0)
            xs = np.minimum(x, sc.n_bodies - 1)
            m = np.linalg.norm(st0[xs, 7:10], axis=1) + sc.radius[xs] * np.linalg.norm(st0[xs, 10:13], axis=1)
            return np.where(ok, m, 0.0)
        terms = (mag(a_i) + mag(b_i)) / (max(9.81, 1.0) * h)
        tol = _feature_tolerance(Fo["feat"], Fo["scale"], h, terms)
        err = np.abs(Fg["feat"].astype(np.float64) - Fo["feat"])
        bad = np.argwhere(err > tol)
        assert bad.size == 0, (bad[:5], Fg["feat"][bad[0][0]], Fo["feat"][bad[0][0]])
        # inverse masses, degrees and depths are exact
        assert np.array_equal(Fg["feat"][:, 7:12].astype(np.float64), Fo["feat"][:, 7:12])
        np.testing.assert_allclose(Fg["scale"], Fo["scale"], rtol=2e-6, atol=0)
        # the plain warm start is what the solve started from
        lam_prev = Fo["feat"][:, 4:7] * Fo["scale"][:, None]
        np.testing.assert_allclose(Fg["lam0"][kind == 0], lam_prev[kind == 0], rtol=2e-6, atol=1e-9)
    finally:
        gpu.close()


def _sim_with_params(theta):
    from paper_2403_17261_gb300 import ovl
    sim = ovl.Simulation(S.resting_sphere())
    sim.mlp_set_params(theta)
    return sim


def test_forward_matches_oracle():
    B = _bounds()
    th = S.mlp_init_params(21, bias_scale=0.3, bf16_exact=True)
    X, _ = S.synthetic_rows(5000, seed=22)
    sim = _sim_with_params(th)
    try:
        np.testing.assert_array_equal(sim.mlp_params(), th)
        y = sim.mlp_forward(X).astype(np.float64)
        y_ref, _ = M.forward(th.astype(np.float64), X.astype(np.float64))
        tol = B.forward_tolerance(th.astype(np.float64), X.astype(np.float64))
        assert np.all(np.abs(y - y_ref) <= tol), float((np.abs(y - y_ref) / tol).max())
        # ragged tails: 1, 15, 17 rows give the same values as within a full batch
        for n in (1, 15, 17):
            np.testing.assert_array_equal(sim.mlp_forward(X[:n]), y[:n].astype(np.float32))
    finally:
        sim.close()


def test_gradient_matches_oracle():
    B = _bounds()
    th = S.mlp_init_params(23, bias_scale=0.3, bf16_exact=True)
    X, T = S.synthetic_rows(3000, seed=24)
    sim = _sim_with_params(th)
    try:
        sim.log_reserve(10000)
        sim.log_append(X, T)
        assert sim.log_size() == 3000
        f, t = sim.log_read(0, 3000)
        assert np.array_equal(f, X) and np.array_equal(t, T)
        for first, count in ((0, 3000), (1000, 777)):
            loss, g = sim.mlp_grad(first, count)
            Xs, Ts = X[first:first + count].astype(np.float64), T[first:first + count].astype(np.float64)
            L_ref, g_ref = M.grad(th.astype(np.float64), Xs, Ts)
            tol = B.grad_tolerance(th.astype(np.float64), Xs, Ts)
            r = np.abs(g.astype(np.float64) - g_ref) / tol
            assert r.max() <= 1.0, (int(r.argmax()), float(r.max()))
            assert abs(loss - L_ref) <= 0.02 * L_ref
            assert abs(sim.mlp_loss(first, count) - L_ref) <= 0.02 * L_ref
    finally:
        sim.close()


def test_adam_first_step_and_training():
    B = _bounds()
    th = S.mlp_init_params(25, bias_scale=0.3, bf16_exact=True)
    X, T = S.synthetic_rows(4096, seed=26)
    sim = _sim_with_params(th)
    try:
        sim.log_reserve(4096)
        sim.log_append(X, T)
        lr = 1e-3
        loss = sim.mlp_train(0, 4096, batch=1024, steps=1, sampling=0, lr=lr)
        th1 = sim.mlp_params().astype(np.float64)
        Xs, Ts = X[:1024].astype(np.float64), T[:1024].astype(np.float64)
        L_ref, g_ref = M.grad(th.astype(np.float64), Xs, Ts)
        tol = B.grad_tolerance(th.astype(np.float64), Xs, Ts)
        ref1, _, _ = M.adam(th.astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS), g_ref, 1, lr=lr)
        # the first Adam step moves every parameter by lr * g / (|g| + eps): by lr
        # in the gradient's direction wherever the gradient is resolved
        sure = np.abs(g_ref) > tol
        assert sure.mean() > 0.5
        np.testing.assert_allclose(th1[sure], ref1[sure], rtol=0, atol=1e-3 * lr + 1e-7)
        assert np.all(np.abs(th1 - th) <= lr * (1 + 1e-3))
        assert abs(loss[0] - L_ref) <= 0.02 * L_ref
        # training lowers the loss on the rows it sees
        before = sim.mlp_loss(0, 4096)
        hist = sim.mlp_train(0, 4096, batch=512, steps=300, sampling=1, lr=3e-3, seed=7)
        after = sim.mlp_loss(0, 4096)
        assert np.all(np.isfinite(hist)) and after < 0.5 * before
    finally:
        sim.close()


def test_graph_replayed_training_matches_single_steps():
    """Calls of 100 or more Adam steps replay a captured CUDA graph of 50
    steps; with every row in every batch, that must equal 100 calls of one
    step launched directly, bit for bit."""
    th = S.mlp_init_params(29, bias_scale=0.2)
    X, T = S.synthetic_rows(2048, seed=30)
    sims = [_sim_with_params(th), _sim_with_params(th)]
    try:
        for sim in sims:
            sim.log_reserve(2048)
            sim.log_append(X, T)
        h_graph = sims[0].mlp_train(0, 2048, batch=2048, steps=120, sampling=0, lr=1e-3)
        h_single = np.concatenate([sims[1].mlp_train(0, 2048, batch=2048, steps=1, sampling=0, lr=1e-3)
                                   for _ in range(120)])
        np.testing.assert_array_equal(sims[0].mlp_params(), sims[1].mlp_params())
        np.testing.assert_array_equal(h_graph, h_single)
        assert h_graph[-1] < h_graph[0]
    finally:
        for sim in sims:
            sim.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_mlp_warm_start_in_a_step(mode):
    from paper_2403_17261_gb300 import ovl
    B, P = _bounds(), _parity()
    sc = S.random_pile(1500, 12, n_sets=5, box=0.3 * 1500 ** (1 / 3) + 1.0)
    th = S.mlp_init_params(27, bias_scale=0.2, bf16_exact=True)
    th[-3] = 1.0   # b3[0]: a positive normal impulse proposal on average
    orc, gpu = P.prepare(sc, warm_steps=2)
    try:
        gpu.mlp_set_params(th)
        gpu.set_warmstart_mode(mode)
        orc.step()
        gpu.step()
        Fo, Fg = orc.features(), gpu.features()
        kind = orc.pairs()["kind"]
        assert np.array_equal(Fo["found"], Fg["found"])
        contact = kind == 0
        use = contact & (~Fo["found"] if mode == 2 else True)
        assert use.sum() > 20
        h = float(sc.scene_dt[0])
        sX = _feature_tolerance(Fo["feat"], Fo["scale"], h) / 6.0   # as standard deviations
        y_tol = B.forward_tolerance(th.astype(np.float64), Fo["feat"], sX)
        mu = float(sc.scene_mu[0])
        lam_ref = M.warm_start(th.astype(np.float64), Fo["feat"], Fo["scale"], np.full(len(kind), mu))
        s = Fo["scale"][:, None]
        tol = s * np.stack([y_tol[:, 0], y_tol[:, 1] + mu * y_tol[:, 0], y_tol[:, 2] + mu * y_tol[:, 0]], axis=1)
        err = np.abs(Fg["lam0"].astype(np.float64) - lam_ref)
        assert np.all(err[use] <= tol[use] + 1e-7), float((err[use] / (tol[use] + 1e-7)).max())
        assert (Fg["lam0"][use, 0] > 0).any()
        # everything else keeps the plain warm start exactly
        keep = ~use
        lam_prev = Fo["feat"][:, 4:7] * Fo["scale"][:, None]
        np.testing.assert_allclose(Fg["lam0"][keep & contact], lam_prev[keep & contact], rtol=2e-6, atol=1e-9)
        st = gpu.stats()
        assert st["device_status"] == 0 and st["phase_ms"].get("warmstart", 0.0) >= 0.0
    finally:
        gpu.close()


def test_log_records_the_solve():
    from paper_2403_17261_gb300 import ovl
    sc = S.pile_small()
    sim = ovl.Simulation(sc)
    try:
        sim.log_reserve(100000)
        sim.log_enable(True)
        for _ in range(3):
            sim.step()
        F = sim.features()
        pr = sim.pairs()
        contact = (pr["key"] >> np.uint64(62)) == 0
        n_last = int(contact.sum())
        total = sim.log_size()
        assert total >= 3 * 600 and n_last > 600
        f, t = sim.log_read(total - n_last, n_last)
        assert np.array_equal(f, F["feat"][contact])
        expect = (pr["lam"][contact] / F["scale"][contact][:, None]).astype(np.float32)
        np.testing.assert_array_equal(t, expect)
        # a full log drops further rows
        sim.log_reserve(1000)
        sim.log_enable(True)
        sim.step()
        sim.step()
        assert sim.log_size() == 1000
    finally:
        sim.close()


def test_mlp_modes_need_parameters():
    from paper_2403_17261_gb300 import ovl
    sim = ovl.Simulation(S.resting_sphere())
    try:
        with pytest.raises(ovl.OvlError):
            sim.set_warmstart_mode(1)
        with pytest.raises(ovl.OvlError):
            sim.features()
    finally:
        sim.close()
