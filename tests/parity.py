"""Helpers for GPU-vs-oracle parity from identical inputs.

``prepare`` runs the FP64 oracle for a few steps, rounds its state and
warm-start impulses to FP32 once, and loads the same rounded values, the same
membership masks and the same step index into both the oracle and a fresh
libovl context -- no input ever comes from the CUDA path.  ``compare_step``
then takes one step on both and checks every record element by element.

Tolerances (FP32 kernel vs FP64 oracle from identical inputs):
  integers (contacts, graph, masks, entries, D, pair order, colours): exact
  velocities, angular velocities:   1e-4 m/s (rad/s), the method's stated bound
  positions:                        1e-5 m
  quaternions:                      1e-5
  contact gap, normal, tangent:     1e-5
  weights:                          1e-6
  impulses:                         the velocity bound x max(1, body mass) (Delta v = Delta lambda / m)

Full-size steps whose PGS is ill-conditioned (the large pile: a +-1 FP32 ulp
change of the inputs moves the FP64 result of a few bodies by ~3e-4 m/s)
pass a ``floor``: the oracle's own algorithm with FP32 sweeps, stepped from
the same inputs.  Its deviation from the FP64 result is what FP32 arithmetic
alone costs on that step, and the CUDA path is held to the plain bound or
FLOOR_FACTOR x that deviation, whichever is larger (positions: plain bound).

Random stress piles (``stress=True``: spheres dropped into overlapping
random positions, so that they meet at up to ~18 m/s with deep penetration)
add 1e-5 x the step's largest speed to the velocity bound: about 170 FP32
unit roundoffs of that speed, which FP32 accumulation over the sweeps of such
impacts can reach.  Every configuration of the method's workloads (the small
pile, the chain, the large pile and the batch) is held to the plain bound.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2403_17261_gb300 import ovl

TOL_V = 1e-4
TOL_V_REL = 1e-5
TOL_X = 1e-5
TOL_Q = 1e-5
TOL_GEOM = 1e-5
TOL_W = 1e-6


def load_identical(orc, gpu):
    """Rounds the oracle's current state and warm-start impulses to FP32 once
    and loads the same rounded values, masks and step index into both sides."""
    st32 = orc.state().astype(np.float32)
    part, key, lam = orc.warmstart()
    lam32 = lam.astype(np.float32)
    orc.set_state(st32.astype(np.float64))
    orc.set_warmstart(part, key, lam32.astype(np.float64))
    gpu.set_membership(orc.masks())
    gpu.set_state(st32)
    gpu.set_warmstart(part, key, lam32)
    gpu.set_step_index(orc.step_index())


def fp32_sweeps_twin(orc, params: dict | None = None):
    """The oracle's algorithm with its PGS sweeps in FP32 (the same source
    built with an FP32 arithmetic type), loaded with the FP64 oracle's
    current inputs: stepped beside it, it measures how far FP32 arithmetic
    alone moves this step's result."""
    twin = O.OracleSim(orc.scene, params, sweeps="f32")
    twin.set_masks(orc.masks())
    twin.set_state(orc.state())
    twin.set_warmstart(*orc.warmstart())
    twin.set_step_index(orc.step_index())
    return twin


def prepare(scene, warm_steps: int = 0, params: dict | None = None, gpu_params: dict | None = None):
    orc = O.OracleSim(scene, params)
    if scene.assign_overlap:
        orc.assign_overlap()
    for _ in range(warm_steps):
        orc.step()
    gp = dict(params or {})
    gp.update(gpu_params or {})
    gpu = ovl.Simulation(scene, gp, partition=False)
    load_identical(orc, gpu)
    return orc, gpu


def _maxabs(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max()) if a.size else 0.0


def _qdist(qa, qb):
    qa = np.asarray(qa, dtype=np.float64)
    qb = np.asarray(qb, dtype=np.float64)
    if not qa.size:
        return 0.0
    d1 = np.abs(qa - qb).max(axis=1)
    d2 = np.abs(qa + qb).max(axis=1)
    return float(np.minimum(d1, d2).max())


FLOOR_FACTOR = 2.0


def _body_max(copies_a, copies_b, entry_ptr, cols):
    d = np.abs(np.asarray(copies_a, np.float64)[:, cols] - np.asarray(copies_b, np.float64)[:, cols]).max(axis=1)
    out = np.zeros(len(entry_ptr) - 1)
    np.maximum.at(out, np.repeat(np.arange(len(entry_ptr) - 1), np.diff(entry_ptr)), d)
    return out


def compare_step(orc, gpu, dt: float = 0.0, iters: int | None = None, check_lambda: bool = True,
                 stress: bool = False, floor=None):
    """One step on both sides; asserts parity of every record; returns a report.

    floor: an FP32-sweep twin of the oracle (fp32_sweeps_twin) from the same
    inputs.  Velocities, quaternions and impulses are then held to the plain
    bound or FLOOR_FACTOR x the twin's own deviation from the FP64 result,
    whichever is larger, and the number of bodies whose copy velocity is off
    by more than the plain bound to FLOOR_FACTOR x the twin's count (+ 10);
    positions keep the plain bound."""
    orc.step(dt, iters)
    gpu.step(dt, iters)
    fl = None
    if floor is not None:
        floor.step(dt, iters)
        ef, eo = floor.entries(), orc.entries()
        sf, so_ = floor.state(), orc.state()
        body_v = _body_max(ef["copies"], eo["copies"], eo["entry_ptr"], slice(7, 13))
        fl = {"copy_v": float(body_v.max()), "v": _maxabs(sf[:, 7:13], so_[:, 7:13]),
              "copy_q": _qdist(ef["copies"][:, 3:7], eo["copies"][:, 3:7]), "q": _qdist(sf[:, 3:7], so_[:, 3:7]),
              "lambda": _maxabs(floor.pairs()["lam"], orc.pairs()["lam"]),
              "over": int((body_v > TOL_V).sum())}
    rep = {}
    sc = orc.scene
    # contacts (Algorithm 1, contact generation)
    ab_o, phi_o, n_o, t_o = orc.contacts()
    ab_g, phi_g, n_g, t_g = gpu.contacts()
    assert ab_o.shape == ab_g.shape, (ab_o.shape, ab_g.shape)
    assert np.array_equal(ab_o, ab_g), "contact pairs differ"
    rep["contacts"] = len(ab_o)
    rep["phi"] = _maxabs(phi_o, phi_g)
    rep["normal"] = _maxabs(n_o, n_g)
    rep["t1"] = _maxabs(t_o, t_g)
    assert rep["phi"] <= TOL_GEOM and rep["normal"] <= TOL_GEOM and rep["t1"] <= TOL_GEOM, rep
    # constraint graph
    rp_o, col_o = orc.graph()
    rp_g, col_g = gpu.graph()
    assert np.array_equal(rp_o, rp_g) and np.array_equal(col_o, col_g), "graph differs"
    # membership after the load balance
    assert np.array_equal(orc.masks(), gpu.membership()), "membership differs"
    # entries, geodesics, weights, copies
    eo, eg = orc.entries(), gpu.entries()
    assert np.array_equal(eo["entry_ptr"], eg["entry_ptr"].astype(np.int64)), "entries differ"
    assert np.array_equal(eo["part"], eg["part"]), "entry workers differ"
    assert np.array_equal(eo["D"], eg["D"]), "geodesic distances differ"
    rep["weight"] = _maxabs(eo["weight"], eg["weight"])
    assert rep["weight"] <= TOL_W, rep
    co, cg = eo["copies"], eg["copies"]
    rep["copy_x"] = _maxabs(co[:, 0:3], cg[:, 0:3])
    rep["copy_q"] = _qdist(co[:, 3:7], cg[:, 3:7])
    rep["copy_v"] = _maxabs(co[:, 7:13], cg[:, 7:13])
    # pairs: worker, key order and colours exact; impulses close
    po, pg = orc.pairs(), gpu.pairs()
    assert np.array_equal(po["part"], pg["part"]), "pair workers differ"
    assert np.array_equal(po["key"], pg["key"]), "pair keys differ"
    assert np.array_equal(po["colour"], pg["colour"]), "colours differ"
    so, sg = orc.state(), gpu.state()
    vmax = float(np.abs(so[:, 7:13]).max()) if so.size else 0.0
    tol_v = TOL_V + (TOL_V_REL * vmax if stress else 0.0)
    rep["tol_v"] = tol_v
    mmax = float(np.max(1.0 / sc.inv_mass[sc.inv_mass > 0])) if np.any(sc.inv_mass > 0) else 1.0
    tol_lam = tol_v * max(1.0, mmax)
    tol_q = {"copy_q": TOL_Q, "q": TOL_Q}
    tol_vv = {"copy_v": tol_v, "v": tol_v}
    if fl is not None:
        rep["floor"] = fl
        tol_lam = max(tol_lam, FLOOR_FACTOR * fl["lambda"])
        tol_q = {k: max(TOL_Q, FLOOR_FACTOR * fl[k]) for k in tol_q}
        tol_vv = {k: max(tol_v, FLOOR_FACTOR * fl[k]) for k in tol_vv}
    rep["lambda"] = _maxabs(po["lam"], pg["lam"])
    if check_lambda:
        assert rep["lambda"] <= tol_lam, rep
    # blended state
    rep["x"] = _maxabs(so[:, 0:3], sg[:, 0:3])
    rep["q"] = _qdist(so[:, 3:7], sg[:, 3:7])
    rep["v"] = _maxabs(so[:, 7:13], sg[:, 7:13])
    body_v = _body_max(cg, co, eo["entry_ptr"], slice(7, 13))
    rep["over"] = int((body_v > TOL_V).sum())
    rep["bodies"] = int(body_v.shape[0])
    assert rep["copy_x"] <= TOL_X and rep["x"] <= TOL_X, rep
    assert rep["copy_q"] <= tol_q["copy_q"] and rep["q"] <= tol_q["q"], rep
    assert rep["copy_v"] <= tol_vv["copy_v"] and rep["v"] <= tol_vv["v"], rep
    if fl is not None:
        assert rep["over"] <= FLOOR_FACTOR * fl["over"] + 10, rep
    return rep
