"""The oracle's threaded loops (contacts per body, PGS per worker, the
geodesic search per body) give the same bits on any thread count."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_17261_gb300 import scenes as S


def _run(make, steps, threads):
    O.set_threads(threads)
    try:
        sc = make()
        sim = O.OracleSim(sc)
        if sc.assign_overlap:
            sim.assign_overlap()
        for _ in range(steps):
            sim.step()
        e = sim.entries()
        return [sim.state(), sim.masks(), sim.pairs()["lam"], sim.pairs()["colour"], e["D"], e["copies"],
                sim.contacts()[0]]
    finally:
        O.set_threads(1)


@pytest.mark.parametrize("make,steps", [
    (lambda: S.pile_large(side=12, n_sets=8), 150),
    (lambda: S.batched(n_scenes=10), 3),
    (lambda: S.random_pile(1500, 12, n_sets=5, box=0.3 * 1500 ** (1 / 3) + 1.0), 3),
])
def test_thread_count_changes_no_bit(make, steps):
    one = _run(make, steps, 1)
    four = _run(make, steps, 4)
    assert one[2].shape[0] > 100
    for a, b in zip(one, four):
        assert a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))
