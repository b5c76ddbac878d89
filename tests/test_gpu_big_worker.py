"""A worker far larger than shared memory holds: 70,560 spheres (a 42 x 42 x
40 lattice, spacing = diameter, jittered, on the ground) all in one worker,
and 134,560 (58 x 58 x 40) in 2 workers split at x = 0, so that both hold
more than 65,534 bodies (worker slots are 32-bit).  The solve takes the global-memory path; one step
from identical inputs matches the FP64 oracle record by record at the
stated bounds (tests/parity.py)."""
import numpy as np
import pytest

from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _lattice(n_sets):
    rng = S.SplitMix64(5)
    side = 42 if n_sets == 1 else 58
    pos = S._lattice_pile(side, side, 40, 1.0, 0.5, 0.01, rng)
    n = pos.shape[0]
    sets = np.zeros(n, np.int32) if n_sets == 1 else (pos[:, 0].astype(np.float32) >= 0).astype(np.int32)
    return S._single("big_worker", pos, np.full(n, 0.5), np.ones(n), [[0, 0, 1, 0]], mu=0.5, dt=1.0 / 60.0,
                     flags=1, gamma=1, beta=4, n_sets=n_sets, set_of_body=sets, iters=10, steps=2, lb_deact_every=1)


@pytest.mark.parametrize("n_sets", [1, 2])
def test_worker_beyond_65534_bodies(n_sets):
    import parity as P
    sc = _lattice(n_sets)
    orc, gpu = P.prepare(sc, warm_steps=0)
    try:
        rep = P.compare_step(orc, gpu)
        ent = gpu.entries()
        per_worker = np.bincount(ent["part"], minlength=n_sets)
        assert per_worker.min() > 65534, per_worker
        assert gpu.stats()["device_status"] == 0
        print(f"\n  {n_sets} worker(s) of {per_worker.tolist()} bodies: {rep['contacts']} contacts, "
              f"|dv| {rep['v']:.2e} m/s, |dx| {rep['x']:.2e} m")
    finally:
        gpu.close()
