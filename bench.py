"""Throughput of the overlapping-partition rigid-body step on GB300.

One "step" is one timestep of Algorithm 1 on the whole workload: contacts,
constraint graph, load balance, membership, colouring, every worker's PGS
solve + integration, geodesic weights and the blend.

Default workload ``pile_large``: 262,144 spheres (64^3 lattice, r ~ U(0.4,0.6),
density 1) dropped into a bowl of four 30-degree planes, 64 k-means workers,
growth depth 2, weight depth 6, 30 PGS sweeps, dt = 1/60, load-balance removals
every 10 steps.  The lattice needs ~130 steps of free fall before it touches
the bowl, so the timed steps start after an untimed settle phase (150 steps by
default) in the contact-rich regime.

Printed (rank 0, one JSON line): body-steps/s over all ranks, the PGS row
iterations/s, a roofline entry for the solver kernel, the FP64 oracle timed on
the host as CPU baseline, an end-to-end figure through the C ABI with host
buffers, SM clocks sampled during the timed region.

``--workload building`` / ``bridge``: box bodies (columns and slabs with two balls; a
jointed plank deck), the stand-ins for Section 6's Building and Two-way Bridge.

``--workload pile_mixed``: 6728 big spheres (radius 1.25, two layers) on the
floor of a box under a 128 x 128 x 16 lattice of small ones (r ~ U(0.4,0.6));
each big sphere takes tens of contacts.  With ``--lb-load contacts`` Algorithm 6 compares loads that
count 1 + contacts per active body instead of bodies (Section 6's proposal);
the line then reports the per-worker row imbalance (max / mean) next to the
throughput.

--impl reference times the FP64 oracle instead (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

# more hardware queues than the library's streams, set before CUDA starts
# (the per-class solve and colouring launches otherwise share queues)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
CONTACT_ROW_BYTES = 84   # per contact per sweep: 60 B read (2 ids, n, t1, lever scalars, k_n, k_t1, k_t2, target, mu) + 12 B lambda read + 12 B lambda write
JOINT_ROW_BYTES = 80     # per joint per sweep: 56 B record (2 slots, r_A, r_B, k[3], target[3]) + 24 B lambda r/w
ENTRY_BYTES = 120        # per (body, worker) per step: 60 B state + params read, 52 B copy write, 8 B index
PAIR_ONCE_BYTES = 24     # per constraint per step: warm-start lambda read + final lambda write
BLEND_ENTRY_BYTES = 53   # per (body, worker) entry: its 52 B copy read + D(o,i) 1 B
BLEND_BODY_BYTES = 64    # per body: 52 B blended state written + 12 B of the start position read
# DRAM bytes (read + write) of every solver launch of one timed step of the
# large pile, from one ncu capture of this file's default command; None until
# a capture matches the current kernel and the timed steps' pair counts.
SOLVE_DRAM_BYTES_PER_STEP = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ovl", choices=["ovl", "reference"])
    ap.add_argument("--workload", default="pile_large",
                    choices=["pile_large", "pile_mixed", "chain", "pile_small", "batched", "building", "bridge",
                             "warmstart", "gamma", "mlp_forward", "mlp_train"],
                    help="warmstart: the learned warm start on the large pile (log, train, "
                         "sweeps to RMS residual 1e-4 against the previous-step warm start); "
                         "mlp_forward: the warm start's network alone on 2^21 rows through ovl_mlp_forward; "
                         "mlp_train: its training alone (Adam, batches of 4096 drawn from 2^20 logged rows) "
                         "through ovl_mlp_train")
    ap.add_argument("--ws-log-steps", type=int, default=6)
    ap.add_argument("--ws-eval-steps", type=int, default=50)
    ap.add_argument("--ws-train-steps", type=int, default=20000)
    ap.add_argument("--settle", type=int, default=None, help="untimed steps before the warm-up")
    ap.add_argument("--lb-load", default="bodies", choices=["bodies", "contacts"],
                    help="load Algorithm 6 compares: active bodies (the paper's) or 1 + contacts per body")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-late-window", dest="late_window", action="store_false",
                    help="skip timing the configuration's last --steps steps")
    return ap.parse_args()


def default_settle(workload):
    return {"pile_large": 150, "pile_mixed": 150, "chain": 0, "pile_small": 0, "batched": 0,
            "building": 0, "bridge": 0, "warmstart": 150, "gamma": 0, "mlp_forward": 0,
            "mlp_train": 0}[workload]


def step_params(ovl, lb_load: str = "bodies") -> dict:
    """Context parameters of the timed step (the full-size parity test uses
    the same ones, so it checks the launch plan this file times)."""
    return dict(flags=ovl.OVL_FLAG_TIMING,
                lb_load=ovl.OVL_LB_CONTACTS if lb_load == "contacts" else ovl.OVL_LB_BODIES)


def make_scene(workload):
    from paper_2403_17261_gb300 import scenes as S
    return S.WORKLOADS[workload]()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (their step times); every rank gets it."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, steps: int, t_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return world * units_per_rank * steps / t_max


def blend_roofline(blend_ms, bytes_blend, steps, peak, peak_kind):
    """HBM roofline of k_blend from the step's own phase timer (events around
    the blend phase, launch included); None if the inputs are unusable."""
    try:
        t = sum(blend_ms) / 1e3
        if t <= 0 or steps <= 0 or not peak:
            return None
        achieved = bytes_blend / t / 1e9
        return {"bound": "hbm", "kernel": "k_blend", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_blend / steps,
                "avg_launch_ms": 1e3 * t / steps, "timer": "phase events around the blend launch"}
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU arm: the FP64 oracle, as it stands, on a bounded sample of the workload
# ---------------------------------------------------------------------------

def host_cores() -> int:
    """Host cores this process may run on (its affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_scene(workload, scene=None):
    """The scene the oracle times, its untimed settle, and a description.  The
    large pile is the benched configuration itself (the oracle settles it)."""
    from paper_2403_17261_gb300 import scenes as S
    if workload in ("pile_large", "warmstart"):
        return (S.pile_large() if scene is None else scene), 150, "the full pile_large configuration (262,144 spheres, 64 workers), settled 150 steps by the oracle itself (untimed)"
    if workload == "pile_mixed":
        return S.pile_mixed(side=16, layers=8, n_sets=16), 150, "pile_mixed generator at 16 x 16 x 8 small + 98 big spheres, 16 k-means workers, settled 150 steps by the oracle itself (untimed)"
    if workload == "chain":
        return S.chain(), 0, "the full 4096-sphere chain"
    if workload == "batched":
        return S.batched(n_scenes=16), 0, "the first 16 of the 512 batched scenes (same generator and seed)"
    if workload == "building":
        return S.box_building(), 0, "the full building (columns, slabs, 2 balls; 16 workers)"
    if workload == "bridge":
        return S.plank_bridge(), 0, "the full plank bridge (1589 planks, 3180 joints; 8 workers)"
    return S.pile_small(), 0, "the full 256-sphere pile"


def oracle_run(workload, steps, warmup, max_seconds=None, params=None, threads=None, single_core_steps=0,
               scene=None):
    """Times the FP64 oracle as it stands on `threads` host threads (default:
    every core of this process), after its own untimed settle.  With
    single_core_steps > 0 the same state is also stepped that many times on
    one thread (the oracle as written, single-threaded)."""
    from oracle import oracle as O
    threads = host_cores() if threads is None else threads
    sc, settle, desc = oracle_sample_scene(workload, scene)
    O.set_threads(threads)
    try:
        sim = O.OracleSim(sc, params)
        if sc.assign_overlap:
            sim.assign_overlap()
        for _ in range(settle + warmup):
            sim.step()
        snap = (sim.state(), sim.masks(), sim.warmstart(), sim.step_index())
        t_total, body_steps, row_iters, done = 0.0, 0, 0, 0
        for k in range(steps):
            t0 = time.perf_counter()
            sim.step()
            t_total += time.perf_counter() - t0
            body_steps += sc.n_bodies
            row_iters += 3 * sim.counts()["pairs"] * sc.iters
            done += 1
            if max_seconds is not None and t_total > max_seconds:
                break
        out = {"value": body_steps / t_total, "row_iters_per_s": row_iters / t_total, "steps": done,
               "seconds": t_total, "cores": threads,
               "sample": desc + f"; steps {snap[3]}..{snap[3] + done - 1} timed after {warmup} warm-up step(s)"}
        if single_core_steps > 0:
            O.set_threads(1)
            sim.set_state(snap[0])
            sim.set_masks(snap[1])
            sim.set_warmstart(*snap[2])
            sim.set_step_index(snap[3])
            t1 = 0.0
            for _ in range(single_core_steps):
                t0 = time.perf_counter()
                sim.step()
                t1 += time.perf_counter() - t0
            out["single_core"] = {"value": sc.n_bodies * single_core_steps / t1, "unit": "body-steps/s",
                                  "cores": 1, "steps": single_core_steps,
                                  "sample": f"the same state, steps {snap[3]}..{snap[3] + single_core_steps - 1}"}
        return out
    finally:
        O.set_threads(1)


def reference_arm(args, rank, world):
    if rank != 0:
        return
    r = oracle_run(args.workload, args.steps, args.warmup, max_seconds=150.0,
                   params=dict(lb_load=1 if args.lb_load == "contacts" else 0))
    line = {
        "impl": "reference", "metric": "body-steps/s", "value": r["value"], "unit": "body-steps/s",
        "n_gpus": args.gpus, "steps": r["steps"], "warmup": args.warmup,
        "ms_per_step": 1e3 * r["seconds"] / max(r["steps"], 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": r["sample"], "host_threads": r["cores"]},
        "cpu_baseline": {"value": r["value"], "unit": "body-steps/s", "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": r["value"], "unit": "body-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "row_iters_per_s": r["row_iters_per_s"],
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def gpu_arm(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import __graft_entry__ as g
    from paper_2403_17261_gb300 import ovl

    torch.cuda.set_device(local_rank)
    g.build()
    sc = make_scene(args.workload)
    stream = torch.cuda.Stream()
    lb_load = ovl.OVL_LB_CONTACTS if args.lb_load == "contacts" else ovl.OVL_LB_BODIES
    sim = ovl.Simulation(sc, step_params(ovl, args.lb_load), stream=stream.cuda_stream)
    settle = default_settle(args.workload) if args.settle is None else args.settle
    # NVTX ranges let a profiler select the timed steps (ncu --nvtx --nvtx-include "timed/")
    torch.cuda.nvtx.range_push("settle")
    for _ in range(settle):
        sim.step()
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("warmup")
    for _ in range(args.warmup):
        sim.step()
    torch.cuda.nvtx.range_pop()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # the end-to-end run below replays the same steps from this snapshot
    snapshot = None if args.no_e2e else (sim.state(), sim.membership(), sim.warmstart(),
                                         sim.step_index_value())
    def time_window(k_steps):
        """k_steps timed steps (L2 flushed before each, outside its interval)."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps)]
        w = dict(solve_ms=[], rows_iters=0, bytes_solve=0.0, launches=[], imbalance=[], blend_ms=[],
                 bytes_blend=0.0, first_step=sim.step_index_value(), pairs=[])
        barrier()
        with ClockSampler(local_rank) as clk:
            for k in range(k_steps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(k))          # L2 flush, outside the timed interval
                    starts[k].record(stream)
                sim.step()
                with torch.cuda.stream(stream):
                    ends[k].record(stream)
                st = sim.stats()
                rows_w = sim.worker_stats()["rows"]
                w["imbalance"].append(float(rows_w.max() / max(rows_w.mean(), 1e-9)))
                w["solve_ms"].append(st["phase_ms"]["solve"])
                w["launches"].append(st["n_launches"])
                n_cons = st["n_pairs"]
                w["pairs"].append(n_cons)
                w["rows_iters"] += st["n_rows"] * sc.iters
                w["bytes_solve"] += (sc.iters * CONTACT_ROW_BYTES * n_cons + PAIR_ONCE_BYTES * n_cons
                                     + ENTRY_BYTES * st["n_entries"])
                w["blend_ms"].append(st["phase_ms"].get("blend", 0.0))
                w["bytes_blend"] += BLEND_ENTRY_BYTES * st["n_entries"] + BLEND_BODY_BYTES * sc.n_bodies
            barrier()
        w["step_ms"] = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        w["clocks"] = clk.summary()
        w["plan"] = np.bincount(sim.solve_plan()).tolist()
        return w

    torch.cuda.nvtx.range_push("timed")
    win = time_window(args.steps)
    torch.cuda.nvtx.range_pop()
    free_b, total_b = torch.cuda.mem_get_info()
    t_max = max_over_ranks(sum(win["step_ms"]) / 1e3, world)
    value = whole_job_rate(world, sc.n_bodies, args.steps, t_max)
    solve_ms, launches, imbalance = win["solve_ms"], win["launches"], win["imbalance"]
    rows_iters, bytes_solve = win["rows_iters"], win["bytes_solve"]
    blend_ms, bytes_blend = win["blend_ms"], win["bytes_blend"]
    solve_s = sum(solve_ms) / 1e3
    last = sim.stats()

    # end to end through the C ABI with host buffers, over the same steps as
    # the timed run (restored from the snapshot): pinned state in, state out
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty((sc.n_bodies, 13), dtype=torch.float32, pin_memory=True).numpy()
        host_out = torch.empty((sc.n_bodies, 13), dtype=torch.float32, pin_memory=True).numpy()
        host_in[:] = snapshot[0]
        sim.set_membership(snapshot[1])
        sim.set_warmstart(*snapshot[2])
        sim.set_step_index(snapshot[3])
        e_s = torch.cuda.Event(enable_timing=True)
        e_e = torch.cuda.Event(enable_timing=True)
        n_e2e = args.steps
        barrier()
        e_s.record(stream)
        for _ in range(n_e2e):
            sim.set_state(host_in)
            sim.step()
            sim.state(out=host_out)
            host_in, host_out = host_out, host_in
        e_e.record(stream)
        barrier()
        te = max_over_ranks(e_s.elapsed_time(e_e) / 1e3, world)
        nbytes = sc.n_bodies * 13 * 4
        e2e = {"value": whole_job_rate(world, sc.n_bodies, n_e2e, te), "unit": "body-steps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": n_e2e}

    # the config's last steps (the overlap has grown under Algorithm 6 by then)
    late = None
    if args.late_window and sc.steps > sim.step_index_value() + args.steps:
        while sim.step_index_value() < sc.steps - args.steps:
            sim.step()
        lw = time_window(args.steps)
        t_late = max_over_ranks(sum(lw["step_ms"]) / 1e3, world)
        late_solve_s = sum(lw["solve_ms"]) / 1e3
        late = {"value": whole_job_rate(world, sc.n_bodies, args.steps, t_late), "unit": "body-steps/s",
                "steps": f"{lw['first_step']}..{lw['first_step'] + args.steps - 1} of {sc.steps}",
                "ms_per_step": 1e3 * t_late / args.steps, "solve_ms_mean": 1e3 * late_solve_s / args.steps,
                "pairs_mean": float(np.mean(lw["pairs"])),
                "solve_effective_gbs": lw["bytes_solve"] / late_solve_s / 1e9,
                "row_iters_per_s": lw["rows_iters"] / late_solve_s,
                "worker_rows_max_over_mean": float(np.mean(lw["imbalance"])),
                "ctas_per_worker_histogram": lw["plan"], "clocks": lw["clocks"]}

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    achieved = bytes_solve / solve_s / 1e9
    if late is not None:
        late["solve_frac_of_peak"] = late["solve_effective_gbs"] / peak
    profile_traffic = SOLVE_DRAM_BYTES_PER_STEP if args.workload == "pile_large" else None
    cpu = None
    if not args.no_cpu_baseline:
        r = oracle_run(args.workload, steps=5, warmup=args.warmup, max_seconds=20.0, params=dict(lb_load=lb_load),
                       single_core_steps=1, scene=sc if args.workload == "pile_large" else None)
        cpu = {"value": r["value"], "unit": "body-steps/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "threads": "workers, bodies and geodesic searches split over the cores",
               "single_core": r.get("single_core")}
    line = {
        "metric": "body-steps/s", "value": value, "unit": "body-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "bodies": sc.n_bodies, "workers": int(np.sum(sc.n_sets)),
                   "pgs_iters": sc.iters, "dt": float(sc.scene_dt[0]), "settle_steps": settle,
                   "l2": "flushed between timed steps (write of 2x L2)",
                   "contacts_last_step": last["n_contacts"], "pairs_last_step": last["n_pairs"],
                   "overlap_bodies_last_step": last["n_overlap"], "max_colours_last_step": last["max_colours"],
                   "lb_load": args.lb_load, "parallelism": f"replicas x{world}"},
        "worker_rows_max_over_mean": float(np.mean(imbalance)),
        "solve_ms_mean": sum(solve_ms) / len(solve_ms),
        "row_iters_per_s": rows_iters / solve_s,
        "phase_ms_last_step": {k: round(v, 4) for k, v in last["phase_ms"].items()},
        "roofline": {"bound": "hbm", "kernel": "k_solve", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": profile_traffic,
                     "achieved_is": "effective: algorithmic bytes (84 B per contact per sweep, 24 B per pair, "
                                    "120 B per entry) / solve time",
                     "dram_frac": (profile_traffic / (solve_s / args.steps) / 1e9 / peak
                                   if profile_traffic else None),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_solve / args.steps,
                     "avg_launch_ms": 1e3 * solve_s / args.steps},
        "blend_roofline": blend_roofline(blend_ms, bytes_blend, args.steps, peak, peak_kind),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(sum(launches)),
        "device_memory_used_gb": round((total_b - free_b) / 1e9, 3),
        "clocks": win["clocks"],
        "ctas_per_worker_histogram": win["plan"],
        "late_window": late,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Learned warm start: sweeps and time to the residual tolerance
# ---------------------------------------------------------------------------

def warmstart_arm(args, rank, world, local_rank):
    """Logs converged impulses (RMS 1e-5 or 1000 sweeps) from plain steps of
    the large pile (seed 2) after it has settled into the bowl, trains the
    network on the GPU, then on a fresh pile (seed 4) compares, step by step
    from identical snapshots, the sweeps and device time the learned and the
    previous-step warm starts need to bring every worker to RMS 1e-4."""
    import torch
    import __graft_entry__ as g
    from paper_2403_17261_gb300 import learned, ovl
    from paper_2403_17261_gb300 import scenes as S

    torch.cuda.set_device(local_rank)
    g.build()
    settle = default_settle("warmstart") if args.settle is None else args.settle
    t0 = time.time()
    log_sim = ovl.Simulation(S.pile_large(seed=2), dict(res_tol=1e-5, res_check_every=5))
    for _ in range(settle):
        log_sim.step()
    sizes = learned.collect(log_sim, steps=args.ws_log_steps, iters=1000, capacity=30_000_000)
    t_log = time.time() - t0
    split = sizes[-2]
    t1 = time.time()
    hist = learned.train(log_sim, split, steps=args.ws_train_steps)
    t_train = time.time() - t1
    held = learned.heldout(log_sim, split, sizes[-1] - split)
    theta = log_sim.mlp_params()
    log_sim.close()

    ev = ovl.Simulation(S.pile_large(seed=4), dict(res_tol=1e-4, res_check_every=1,
                                                   flags=ovl.OVL_FLAG_TIMING | ovl.OVL_FLAG_RESIDUAL))
    ev.mlp_set_params(theta)
    for _ in range(settle):
        ev.step()
    with ClockSampler(local_rank) as clk:
        r = learned.compare(ev, steps=args.ws_eval_steps)
    ev.close()
    if rank != 0:
        return
    mlp, prev = r[ovl.OVL_WS_MLP], r[ovl.OVL_WS_PREVIOUS]

    def summary(x):
        return {"sweeps_sum_over_workers": float(x["sweeps"].mean()),
                "sweeps_max_worker": float(x["max_sweeps"].mean()),
                "solve_ms": float(x["solve_ms"].mean()), "warmstart_ms": float(x["warmstart_ms"].mean()),
                "step_ms": float(x["step_ms"].mean()), "steps_all_workers_converged": int(x["converged"].sum()),
                "residual_rms": float(x["residual_rms"].mean())}

    line = {
        "metric": "PGS sweeps to RMS residual <= 1e-4 (learned warm start)",
        "value": float(mlp["sweeps"].mean()), "unit": "sweeps/step (sum over workers)",
        "higher_is_better": False, "n_gpus": 1, "steps": args.ws_eval_steps, "warmup": settle,
        "vs_baseline": None, "dtype": "f32 solve, bf16 network", "data": "synthetic",
        "config": {"workload": "pile_large 262,144 spheres, 64 workers: logged on seed 2, evaluated on seed 4",
                   "settle_steps": settle, "log_steps": args.ws_log_steps, "log_rows": sizes[-1],
                   "train_rows": split, "train_steps": args.ws_train_steps, "batch": 4096, "lr": 1e-3,
                   "eval_tolerance": 1e-4, "sweep_cap": 1000},
        "learned": summary(mlp), "previous_step": summary(prev),
        "sweeps_ratio_learned_over_previous": float(mlp["sweeps"].mean() / prev["sweeps"].mean()),
        "solve_time_ratio_learned_over_previous": float((mlp["solve_ms"] + mlp["warmstart_ms"]).mean() / prev["solve_ms"].mean()),
        "heldout_mse": held, "train_loss_last": float(np.mean(hist[-100:])),
        "seconds": {"log": t_log, "train": t_train},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def mlp_forward_arm(args, rank, world, local_rank):
    """The learned warm start's network alone (the tensor-core inference
    kernel): 2^21 rows of 12 seeded features with seeded parameters through
    ovl_mlp_forward, host arrays in and out; rows per second over --steps
    calls after --warmup."""
    import time
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_2403_17261_gb300 import ovl
    from paper_2403_17261_gb300 import scenes as S

    torch.cuda.set_device(local_rank)
    g.build()
    sim = ovl.Simulation(S.pile_small(), {})
    rng = np.random.default_rng(7)
    sim.mlp_set_params((rng.standard_normal(ovl.OVL_MLP_N_PARAMS) * 0.1).astype(np.float32))
    n = 1 << 21
    feat = rng.standard_normal((n, 12)).astype(np.float32)
    for _ in range(args.warmup):
        sim.mlp_forward(feat)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y = sim.mlp_forward(feat)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    sim.close()
    if rank == 0:
        print(json.dumps({"metric": "network rows/s", "value": n / dt, "unit": "rows/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                          "data": "synthetic", "config": {"workload": "mlp_forward", "rows": n,
                                                          "network": "12-64-64-3 ReLU"},
                          "e2e": {"value": n / dt, "unit": "rows/s", "h2d_bytes_per_step": n * 64,
                                  "d2h_bytes_per_step": n * 12},
                          "y0": [float(v) for v in y[0]]}), flush=True)


def mlp_train_arm(args, rank, world, local_rank):
    """The learned warm start's training alone (forward and backward passes,
    tensor-core weight gradients, Adam): 2^20 seeded rows in the context's
    log, then per step one ovl_mlp_train call of 500 Adam steps on batches of
    4096 rows drawn with replacement; training rows per second over --steps
    calls after --warmup (each call returns its per-step losses to the host)."""
    import time
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_2403_17261_gb300 import ovl
    from paper_2403_17261_gb300 import scenes as S

    torch.cuda.set_device(local_rank)
    g.build()
    sim = ovl.Simulation(S.pile_small(), {})
    n, batch, adam_steps = 1 << 20, 4096, 500
    X, T = S.synthetic_rows(n, seed=8)
    sim.log_reserve(n)
    sim.log_append(X, T)
    sim.mlp_set_params(S.mlp_init_params(9))
    for k in range(args.warmup):
        sim.mlp_train(0, n, batch, adam_steps, seed=k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        loss = sim.mlp_train(0, n, batch, adam_steps, seed=100 + k)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    sim.close()
    if rank == 0:
        rows = batch * adam_steps
        print(json.dumps({"metric": "training rows/s", "value": rows / dt, "unit": "rows/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                          "data": "synthetic", "config": {"workload": "mlp_train", "logged_rows": n,
                                                          "batch": batch, "adam_steps_per_call": adam_steps,
                                                          "network": "12-64-64-3 ReLU"},
                          "e2e": {"value": rows / dt, "unit": "rows/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 4 * adam_steps},
                          "final_loss": float(np.asarray(loss).reshape(-1)[-1])}), flush=True)


def gamma_arm(args, rank, world, local_rank):
    """Growth depth sweep and computed-versus-uniform weights on a hanging
    chain of 512 links in 8 workers, 1000 sweeps (the paper's error-study
    setting): from 20 states of a single-worker run, one partitioned step per
    configuration; the joint violation it adds over the single-worker step
    (per chain length) and the largest velocity deviation."""
    import torch
    import __graft_entry__ as g
    from paper_2403_17261_gb300 import experiments

    torch.cuda.set_device(local_rank)
    g.build()
    with ClockSampler(local_rank) as clk:
        r = experiments.partition_error()
    if rank != 0:
        return
    default = next(t for t in r["runs"] if t["gamma"] == 2 and t["weights"] == "geodesic")
    line = {
        "metric": "joint violation added by partitioning in one step / chain length",
        "value": default["added_violation_over_length"], "unit": "m/m", "higher_is_better": False,
        "n_gpus": 1, "steps": r["samples"], "warmup": 0, "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"chain {r['chain_links']} spheres, {r['workers']} workers, {r['sweeps']} sweeps, "
                               "dt 1/120; value at gamma 2, geodesic weights"},
        "sweep": r["runs"], "single_worker_violation_over_length": r["single_worker_violation_over_length"],
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "warmstart":
        warmstart_arm(args, rank, world, local_rank)
        return
    if args.workload == "gamma":
        gamma_arm(args, rank, world, local_rank)
        return
    if args.workload == "mlp_forward":
        mlp_forward_arm(args, rank, world, local_rank)
        return
    if args.workload == "mlp_train":
        mlp_train_arm(args, rank, world, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    gpu_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
