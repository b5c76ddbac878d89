"""The growth-depth sweep and the weights comparison run end to end on the
GPU: overlap grows with gamma, and from the same states the geodesic weights
of Eq 15-16 add less joint violation and velocity error in one partitioned
step than uniform weights (the oracle gives 1.3e-6 against 3.0e-6 of the
chain's length and 0.023 against 0.054 m/s at gamma 2 on this chain)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_partition_error_small(capsys):
    from paper_2403_17261_gb300 import experiments
    r = experiments.partition_error(gammas=(0, 2, 4), samples=8)
    runs = r["runs"]
    assert len(runs) == 6
    for run in runs:
        assert np.isfinite(run["added_violation_over_length"]) and np.isfinite(run["velocity_deviation_max"])
    geo = {run["gamma"]: run for run in runs if run["weights"] == "geodesic"}
    uni = {run["gamma"]: run for run in runs if run["weights"] == "uniform"}
    assert geo[0]["overlap_bodies"] < geo[2]["overlap_bodies"] < geo[4]["overlap_bodies"]
    for g in (2, 4):
        assert geo[g]["velocity_deviation_max"] < uni[g]["velocity_deviation_max"]
        assert geo[g]["added_violation_over_length"] < uni[g]["added_violation_over_length"]
    with capsys.disabled():
        print("\n  gamma  weights   overlap  added violation/length  max |dv|")
        for run in runs:
            print(f"  {run['gamma']:5d}  {run['weights']:8s}  {run['overlap_bodies']:7d}"
                  f"  {run['added_violation_over_length']:.3e}  {run['velocity_deviation_max']:.3e}")
