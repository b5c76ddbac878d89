"""The growth-depth sweep and the computed-versus-uniform weights comparison
(Section 5.1, Figure 6; Section 5.3, Figure 8), measured on the GPU.

The paper shows that a larger growth depth gamma shares more bodies between
workers and narrows the gaps that open at joints near partition interfaces,
and that weights from graph geodesics (Eq 15-16) remove errors that uniform
weights leave.  Long runs of a hanging chain cannot separate that error from
the solver's own (a chain of 512 links keeps about 0.4 % of its length in
joint gaps even with one worker and 1000 sweeps) and from the divergence of
chaotic trajectories.  So ``partition_error`` measures what partitioning adds
in one step: a single-worker run of the chain supplies the states; from each
sampled state every configuration (gamma, weighting) takes one partitioned
step, and it is compared with the single-worker step from the same state:

- added joint violation: the pivot gaps after the partitioned step minus
  those after the single-worker step, summed over joints, over the chain's
  length (Section 6's position-level measure);
- velocity deviation: the largest |v| difference over bodies.

Argument marshalling only: every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import ovl
from . import scenes as S


def partition_error(gammas=(0, 1, 2, 3, 4, 6), n: int = 512, n_sets: int = 8, iters: int = 1000,
                    samples: int = 20, every: int = 5, settle: int = 20, seed: int = 1) -> dict:
    """Both weightings at every gamma (weight search depth 2 gamma + 2)."""
    ref_sc = S.chain(seed=seed, n=n, n_sets=1, iters=iters)
    length = (n + 1) * float(ref_sc.meta["link_length"])
    ref = ovl.Simulation(ref_sc)
    weightings = (ovl.OVL_WEIGHTS_GEODESIC, ovl.OVL_WEIGHTS_UNIFORM)
    sims = {(g, w): ovl.Simulation(S.chain(seed=seed, n=n, n_sets=n_sets, gamma=g, iters=iters),
                                   dict(weights=w, flags=ovl.OVL_FLAG_TIMING))
            for g in gammas for w in weightings}
    rec = {key: {"dj": [], "dv": [], "ms": [], "overlap": 0} for key in sims}
    ref_violation = []
    try:
        for k in range(settle + samples * every):
            sample = k >= settle and (k - settle) % every == 0
            s0 = ref.state() if sample else None
            ref.step(iters=iters)
            if not sample:
                continue
            s1 = ref.state()
            j_ref = ref.joint_error()["sum"]
            ref_violation.append(j_ref / length)
            for key, sim in sims.items():
                sim.set_state(s0)
                sim.step(iters=iters)
                st = sim.stats()
                r = rec[key]
                r["dj"].append((sim.joint_error()["sum"] - j_ref) / length)
                r["dv"].append(float(np.abs(sim.state()[:, 7:10] - s1[:, 7:10]).max()))
                r["ms"].append(st["phase_ms"]["total"])
                r["overlap"] = st["n_overlap"]
    finally:
        ref.close()
        for sim in sims.values():
            sim.close()
    runs = []
    for (g, w), r in rec.items():
        runs.append({
            "gamma": g, "beta": 2 * g + 2, "weights": "uniform" if w else "geodesic",
            "overlap_bodies": int(r["overlap"]),
            "added_violation_over_length": float(np.mean(r["dj"])),
            "velocity_deviation_max": float(np.mean(r["dv"])),
            "step_ms": float(np.mean(r["ms"])),
        })
    return {"runs": runs, "chain_links": n, "workers": n_sets, "sweeps": iters, "samples": samples,
            "single_worker_violation_over_length": float(np.mean(ref_violation))}
