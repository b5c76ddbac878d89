"""Workflow of the learned warm start on top of the C ABI.

1. ``collect``: run the plain method with a tight residual tolerance and log
   every contact's features with the impulses its solve ended with.
2. ``train``: fit the 12-64-64-3 network on the GPU (the library's own
   forward, backward and Adam kernels).
3. ``heldout``: mean squared error, on logged steps the network did not see,
   of the network's proposal and of the previous-step impulses (the plain
   warm start), both against the impulses the solver converged to.
4. ``compare``: on fresh steps, the PGS sweeps and device time each warm
   start needs to bring every worker's RMS complementarity residual to the
   tolerance, from the same state, membership and impulse history.

Argument marshalling only: every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import ovl
from . import scenes as S


def collect(sim: ovl.Simulation, steps: int, iters: int = 1000, capacity: int = 20_000_000) -> list[int]:
    """Steps ``sim`` with the log on; returns the log size after each step.
    Create ``sim`` with the tolerance the targets should meet (res_tol)."""
    if sim.log_size() == 0:
        sim.log_reserve(capacity)
    sim.log_enable(True)
    sizes = []
    for _ in range(steps):
        sim.step(iters=iters)
        sizes.append(sim.log_size())
    sim.log_enable(False)
    return sizes


def train(sim: ovl.Simulation, n_rows: int, steps: int = 20000, batch: int = 4096, lr: float = 1e-3,
          seed: int = 1, init_seed: int = 5) -> np.ndarray:
    """Trains a fresh network (last layer zero: it starts as the plain warm
    start) on log rows [0, n_rows); returns the per-step batch losses."""
    sim.mlp_set_params(S.mlp_init_params(init_seed, zero_output=True))
    return sim.mlp_train(0, n_rows, batch=batch, steps=steps, sampling=1, lr=lr, seed=seed)


def heldout(sim: ovl.Simulation, first: int, count: int) -> dict:
    """MSE of the network and of the previous-step impulses on log rows
    [first, first + count), in the network's scaled units."""
    f, t = sim.log_read(first, count)
    prev = float(np.mean((f[:, 4:7].astype(np.float64) - t.astype(np.float64)) ** 2))
    return dict(mlp=sim.mlp_loss(first, count), previous=prev, rows=count)


def compare(sim: ovl.Simulation, steps: int, modes=(ovl.OVL_WS_MLP, ovl.OVL_WS_PREVIOUS),
            iters: int = 1000) -> dict:
    """Runs every step once per mode from the same snapshot; the trajectory
    continues from the last mode's result.  ``sim`` needs res_tol set,
    res_check_every = 1 and OVL_FLAG_TIMING | OVL_FLAG_RESIDUAL.  Returns,
    per mode, arrays over the steps: sweeps summed over workers, the most
    sweeps of one worker, solve and warm-start device milliseconds, whole-step
    milliseconds, the final RMS residual and whether every worker reached
    the tolerance."""
    out = {m: {k: [] for k in ("sweeps", "max_sweeps", "solve_ms", "warmstart_ms", "step_ms",
                               "residual_rms", "converged")} for m in modes}
    tol = float(sim.params.res_tol)
    for _ in range(steps):
        snap = (sim.state(), sim.membership(), sim.warmstart(), sim.step_index_value())
        for i, mode in enumerate(modes):
            if i:
                sim.set_state(snap[0])
                sim.set_membership(snap[1])
                sim.set_warmstart(*snap[2])
                sim.set_step_index(snap[3])
            sim.set_warmstart_mode(mode)
            sim.step(iters=iters)
            st, ws = sim.stats(), sim.worker_stats()
            r = out[mode]
            r["sweeps"].append(int(ws["iters"].sum()))
            r["max_sweeps"].append(int(ws["iters"].max()))
            r["solve_ms"].append(st["phase_ms"]["solve"])
            r["warmstart_ms"].append(st["phase_ms"]["warmstart"])
            r["step_ms"].append(st["phase_ms"]["total"])
            r["residual_rms"].append(st["residual_rms"])
            rms_w = np.sqrt(ws["res_sq"] / np.maximum(ws["rows"], 1))
            r["converged"].append(bool(np.all(rms_w <= tol * (1 + 1e-6))))
    sim.set_warmstart_mode(ovl.OVL_WS_PREVIOUS)
    return {m: {k: np.asarray(v) for k, v in r.items()} for m, r in out.items()}
