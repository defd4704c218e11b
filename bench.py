#!/usr/bin/env python
"""Throughput of the implicit DER step (DisMech, arXiv 2311.18126) on GB300.

One step = one backward-Euler time step of every rod of the batch: Newton's
method to the 1e-10 scaled residual, with every phase (frames, stretch,
bend-twist gradients/Hessians, assembly, banded solve, commit) in the CUDA
library.  Workload: 4096 independent clamped rods, N ~ U{20..200} nodes,
L ~ U(0.2, 1.5) m, h ~ U(5e-4, 3e-3) m, log10 E ~ U(6, 8), natural
curvature ~ U[-5, 5]^2 1/m, gravity, damping 0.1, dt = 1e-3 s (synthetic,
seeded; the same generator the parity tests use).

Multi-GPU: rods are independent, so each rank runs its own seeded batch of
4096 rods with no collective on the data path (weak scaling); the barrier
and the max over ranks bracket the timed region only.

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rod-steps/s at 1e-10 Newton residual, batched; learned vs plain speedup; % roofline"
UNIT = "rod-steps/s"
WORKLOAD = "uneven_rods: 4096 clamped rods, N~U{20..200}, dt=1e-3 s, backward Euler, FP64"

# FP64 flops executed per work unit of each kernel (DADD + DMUL + 2 DFMA,
# predicated-on lanes), counted by ncu on the uneven-rods workload
# (profiles/kernel_fp64_counts.json); the denominator is the measured FP64
# FMA throughput of the device.
FP64_FLOPS_PER_UNIT = {
    "bend_twist_gradient": None,
    "bend_twist_hessian": None,
    "edge_frames_stretch": None,
    "residual_rows": None,
    "jacobian_band_rows": None,
    "band_ldlt_solve": None,
    "bend_twist_fused": None,
    "residual_jacobian_rows": None,
}
UNIT_NAME = {"bend_twist_gradient": "stencil", "bend_twist_hessian": "stencil",
             "limb_schur_solve": "DOF", "ground_contact_friction": "node",
             "contact_band_lu": "flop of the trailing updates",
             "residual_rows_general": "DOF row", "assemble_general": "DOF",
             "edge_frames_stretch": "edge", "residual_rows": "DOF row",
             "jacobian_band_rows": "DOF row", "band_ldlt_solve": "DOF",
             "bend_twist_fused": "stencil", "residual_jacobian_rows": "DOF row",
             "step_begin": "DOF", "step_commit": "DOF"}


def _hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("hbm_gbs", 6800.0))
    return 6800.0  # fallback figure of an earlier GB300 measurement


HBM_PEAK = _hbm_peak()


def _load_counts():
    p = os.path.join(ROOT, "profiles", "kernel_fp64_counts.json")
    if os.path.exists(p):
        d = json.load(open(p))
        for k, v in d.get("flops_per_unit", {}).items():
            FP64_FLOPS_PER_UNIT[k] = v


def launch_shapes(sysm, args):
    """Launch shapes: given (--tuning, a dict of autotune's fields), the
    defaults (--no-autotune), or measured by the autotuner."""
    if args.tuning:
        t = json.loads(args.tuning)
        sysm.set_tuning(t)
        return dict(t, source="given")
    return None if args.no_autotune else sysm.autotune(steps=2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rods", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="uneven_rods",
                    choices=["uneven_rods", "star_robots", "coil", "gripper", "long_rods",
                             "warm_start",
                             "warm_start_rods", "calibration", "mlp"],
                    help="uneven_rods: the headline batch (default); star_robots: limbed "
                         "robots on the ground with a gait; coil: edge-edge self-contact; "
                         "long_rods: 64 rods of 4000-6000 nodes, partitioned vs sequential "
                         "band solve; "
                         "gripper: five 60-node fingers entangling with frictional contact "
                         "between them; "
                         "warm_start: learned vs extrapolated Newton guess on star robots; "
                         "warm_start_rods: the same on the headline batch of uneven rods; "
                         "calibration: adjoint gradient of a 500-step star-robot rollout; "
                         "mlp: the warm-start network's tensor-core inference and training "
                         "at the headline batch's segment count")
    ap.add_argument("--robots", type=int, default=1024)
    ap.add_argument("--predictor", default="projected", choices=["extrapolate", "projected"],
                    help="Newton's starting guess on single rods: q_n + dt qdot_n, or that "
                         "guess with every edge rescaled to its committed length")
    ap.add_argument("--integrator", default="be", choices=["be", "midpoint"],
                    help="backward Euler (default) or implicit midpoint (Sec. III-C)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes")
    ap.add_argument("--split-first", action="store_true",
                    help="run a step's first Newton round with the split passes (for "
                         "counting the split kernels with every unit active)")
    ap.add_argument("--rows", type=int, default=0,
                    help="mlp workload: rows of the inference batch (a multiple of 128; "
                         "default the 444544 segments of the 4096-rod batch)")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes to apply instead of autotuning (JSON object with the "
                         "fields of the 'autotune' key of an earlier line), e.g. for profiler "
                         "launch lists in the bench's own launch configuration")
    return ap.parse_args()


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_of_batch(make, ws, rank):
    """This rank's shard of one seeded batch: ``make(ws)`` builds the batch
    for ws ranks (ws times the one-GPU size: weak scaling) as (desc, params,
    per-rod controls); it is split into contiguous ranges of whole systems
    balanced by DOF count, one per rank (no exchange inside a step).
    Returns the rank's (desc, params, controls, rods of the whole batch).
    ``controls`` is an array of rows per interior node, or a gait dict of
    per-rod arrays, or None."""
    from paper_2311_18126_gb300 import shard
    desc, params, ctl = make(ws)
    parts = shard.partition(desc, ws)
    b, e = parts[rank]
    sub = shard.sub_descriptor(desc, b, e)
    if isinstance(ctl, dict):  # a gait: per-rod arrays, robot ids renumbered
        ctl = {k: (np.asarray(v)[b:e] if np.ndim(v) == 1 and len(v) == len(desc["nodes_per_rod"])
                   else v) for k, v in ctl.items()}
    elif ctl is not None:
        k0, k1 = shard.kbar_ranges(desc, parts)[rank]
        ctl = ctl[k0:k1]
    return sub, params, ctl, len(desc["nodes_per_rod"])


def max_over_ranks(x, ws, device=None):
    """Largest value of x over the ranks (the timed region ends when the
    slowest rank ends); x unchanged on one rank."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_rate(total_rods, steps, seconds):
    """Whole-job rod-steps per second: the rods of all ranks over the
    slowest rank's time."""
    return total_rods * steps / seconds


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first
        # sample so that the timed region that follows is sampled throughout
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[2][k].lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def _oracle_worker(job):
    """One pool process: the oracle on its rods of the uneven-rods batch
    (regenerated from its seed), one torch thread; returns the seconds of
    the timed steps, the rods and their nodes."""
    n_rods, params, rods, warmup, steps = job
    import torch
    torch.set_num_threads(1)
    import workloads
    from oracle import OracleSystems
    desc, _, kbar = workloads.uneven_rods(n_rods=n_rods, seed=2)
    sub, kb = workloads.subset(desc, rods, kbar)
    o = OracleSystems(sub, params)
    o.set_natural_curvature(0, len(rods), kb)
    for _ in range(warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(steps):
        out = o.step(1)
        assert all(x[0] == 0 for x in out), out
    return time.perf_counter() - t0, len(rods), int(np.sum(np.asarray(sub["nodes_per_rod"])))


def oracle_pool_rate(n_rods, params, rods, warmup, steps, cores=None):
    """The CPU oracle on the host cores: one process per core (spawned, one
    torch thread each), the sampled rods dealt round-robin, every process
    stepping its rods `warmup` untimed and `steps` timed steps.  Returns
    (rod-steps/s = all timed rod-steps / the slowest process's time, that
    time, processes, nodes)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    cores = max(1, min(cores, len(rods)))
    jobs = [(n_rods, params, [int(r) for r in rods[k::cores]], warmup, steps)
            for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    tmax = max(r[0] for r in res)
    return sum(r[1] for r in res) * steps / tmax, tmax, cores, sum(r[2] for r in res)


def sample_rods(n_total, k, seed=12345):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=k, replace=False))


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return
    import workloads
    desc, params, kbar = workloads.uneven_rods(n_rods=args.rods, seed=2)
    params = dict(params, integrator=args.integrator)
    if args.integrator == "midpoint":
        params["line_search"] = True
    cores = os.cpu_count() or 1
    rods = sample_rods(args.rods, 2 * cores)
    v, dt, used, nodes = oracle_pool_rate(args.rods, params, rods, args.warmup, args.steps, cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.integrator == "be" else
                       WORKLOAD.replace("backward Euler", "implicit midpoint"),
                       "rods_per_step": len(rods),
                       "sample": "rods %s of the 4096 (seeded), consecutive steps" % rods.tolist()},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": "%d seeded rods (%d nodes) of the 4096-rod batch dealt "
                                       "over %d single-threaded oracle processes, %d timed "
                                       "steps after %d untimed" %
                                       (len(rods), nodes, used, args.steps, args.warmup)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args):
    import torch
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads
    from paper_2311_18126_gb300 import System, ensure_built, fp64_peak_gflops
    ensure_built()
    _load_counts()
    desc, params, kbar, R_all = shard_of_batch(
        lambda n: workloads.uneven_rods(n_rods=args.rods * n, seed=2), ws, rank)
    params = dict(params, integrator=args.integrator)
    if args.integrator == "midpoint":
        # without numerical damping plain Newton diverges on stiff rods of
        # this batch (the oracle likewise, e.g. rod 379 at its 5th step)
        params["line_search"] = True
    params["predictor"] = args.predictor
    R = len(desc["nodes_per_rod"])
    sysm = System(desc, params)
    if args.split_first:
        sysm.set_fused_first(False)
    sysm.set_natural_curvature(0, R, kbar)
    peak_fp64 = fp64_peak_gflops()

    def barrier():
        if ws > 1:
            import torch.distributed as tdist
            tdist.barrier()

    tuning = launch_shapes(sysm, args)
    for _ in range(args.warmup):
        sysm.step(1, stats=False)
    torch.cuda.synchronize()
    snap = _snapshot(sysm)
    sysm.set_profiling(False)  # counters reset; Newton rounds run as CUDA graphs
    barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters = []
    e0.record()
    for _ in range(args.steps):
        st = sysm.step(1, stats=True)
        iters.append(sysm.iterations.copy())
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    n_launch = sum(v[0] for v in sysm.get_profile().values())
    tmax = max_over_ranks(ms, ws, "cuda")
    value = job_rate(R_all, args.steps, tmax * 1e-3)
    # the same steps again from the same state with the host driving the
    # rounds, then a profiled pass (per-kernel CUDA events, host-driven) for
    # the kernel table
    _restore(sysm, snap)
    host_ms, _, _ = _timed_steps(sysm, args.steps, None, 0, local, graphs=False, clocks=False)
    _restore(sysm, snap)
    sysm.set_profiling(True)
    _timed_steps(sysm, args.steps, None, 0, local, clocks=False)
    prof = sysm.get_profile()
    sysm.set_profiling(False)

    # end to end through the public API with pinned host buffers
    n = sysm.n_state
    hq = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hv = torch.empty(n, dtype=torch.float64, pin_memory=True)
    q0, v0 = sysm.get_state()
    hq.numpy()[:] = q0
    hv.numpy()[:] = v0
    barrier()
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    nq, nv = hq.numpy(), hv.numpy()
    for _ in range(e2e_steps):
        sysm.set_state(nq, nv)              # host -> device from pinned buffers
        sysm.step(1, stats=False)
        sysm.get_state(nq, nv)              # device -> host into the same buffers
    torch.cuda.synchronize()
    te = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
    e2e = {"value": job_rate(R_all, e2e_steps, te), "unit": UNIT,
           "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": 2 * n * 8}

    # dominant kernel and its FP64 roofline
    dom = max(prof, key=lambda k: prof[k][2])
    launches, units, kms = prof[dom]
    per_launch_ms = kms / launches
    fpu = FP64_FLOPS_PER_UNIT.get(dom)
    roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s",
            "peak": peak_fp64 / 1e3, "peak_source": "measured FP64 FMA throughput "
            "(dm_fp64_peak_gflops, this run)", "traffic": None}
    if fpu:
        ach = fpu * units / launches / (per_launch_ms * 1e-3) / 1e12
        roof.update({"achieved": ach, "frac": ach / (peak_fp64 / 1e3),
                     "flops_per_unit": fpu, "unit_name": UNIT_NAME.get(dom),
                     "units_per_launch": units / launches})
        if dom == "band_ldlt_solve":
            # the executed count includes the lanes' redundant work (the
            # reciprocal by all eight lanes of a chain, idle multiplier
            # lanes); the LDL^T's own arithmetic per eliminated column and
            # its back-substitution row is 10 multipliers, 55 symmetric
            # updates, 10 right-hand-side updates, the reciprocal and z_j,
            # and 10 updates: 162 flops, plus about 730 per rod for the
            # 10 x 10 separator
            nr = 4 * np.asarray(desc["nodes_per_rod"], dtype=np.float64) - 1
            own = float((162.0 * (nr - 10) + 730.0).sum() / nr.sum())
            roof.update({"own_flops_per_unit": round(own, 1),
                         "frac_own_flops": ach * own / fpu / (peak_fp64 / 1e3)})
    else:
        roof.update({"achieved": None, "frac": None})
    counts = os.path.join(ROOT, "profiles", "kernel_fp64_counts.json")
    if os.path.exists(counts):
        tr = json.load(open(counts)).get("dram_bytes_per_unit", {}).get(dom)
        if tr:
            roof["traffic"] = tr * units / launches
    kernels = {k: {"launches": v[0], "units": v[1], "ms_total": round(v[2], 3),
                   "share": round(v[2] / sum(x[2] for x in prof.values()), 4)}
               for k, v in prof.items()}
    # every kernel with counted FP64 work: achieved FP64 rate and fraction of
    # the measured FP64 peak, and DRAM rate from the counted bytes per unit
    bpu = {}
    if os.path.exists(counts):
        bpu = json.load(open(counts)).get("dram_bytes_per_unit", {})
    for k, v in prof.items():
        f = FP64_FLOPS_PER_UNIT.get(k)
        if f and v[2] > 0:
            rate = f * v[1] / (v[2] * 1e-3) / 1e12
            kernels[k]["fp64_tflops"] = round(rate, 4)
            kernels[k]["fp64_frac"] = round(rate / (peak_fp64 / 1e3), 4)
        if bpu.get(k) and v[2] > 0:
            gbs = bpu[k] * v[1] / (v[2] * 1e-3) / 1e9
            kernels[k]["dram_gbs"] = round(gbs, 1)
            kernels[k]["hbm_frac"] = round(gbs / HBM_PEAK, 4) if HBM_PEAK else None

    it = np.array(iters)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.integrator == "be" else
                       WORKLOAD.replace("backward Euler", "implicit midpoint"), "rods_per_gpu": R,
                       "nodes_per_gpu": int(np.sum(desc["nodes_per_rod"])),
                       "dofs_per_gpu": int(n), "dt": params["dt"], "newton_tol": params["tol"],
                       "line_search": bool(params.get("line_search", False)),
                       "predictor": params.get("predictor", "extrapolate"),
                       "first_round": "split" if args.split_first else "fused",
                       "parallelism": "dp%d: each GPU steps a DOF-balanced shard of contiguous systems of one batch %d x the one-GPU size" % (ws, ws),
                       "l2": "no flush: per-iteration working set (~0.7 GB) exceeds L2"},
            "newton": {"iters_mean": float(it.mean()), "iters_max": int(it.max()),
                       "node_steps_per_s": value * float(np.mean(desc["nodes_per_rod"]))},
            "clocks": clocks, "e2e": e2e,
            "gpu_launches": int(n_launch),
            "rounds": {"mode": "one CUDA graph per step (device-side while loop over Newton "
                               "rounds)", "host_loop_ms_per_step": host_ms / args.steps,
                       "note": "host loop timed on the same steps from the same state"},
            "autotune": tuning,
            "kernel_timing": "per-kernel CUDA events in a separate pass of the same number "
                             "of steps right after the timed region (host-driven rounds, "
                             "same kernels and launch shapes)",
            "roofline": roof, "kernels": kernels}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rods = sample_rods(R, 2 * cores)
        v, dt, used, nodes = oracle_pool_rate(R, params, rods, 0, 5, cores)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": "%d seeded rods (%d nodes) of the batch dealt over "
                                          "%d single-threaded oracle processes, 5 steps from "
                                          "the initial state, %.1f s" % (len(rods), nodes, used,
                                                                         dt)}
    if rank == 0:
        print(json.dumps(line))
    sysm.close()
    if ws > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def _snapshot(sysm):
    q, v = sysm.get_state()
    d1, beta = sysm.get_frames()
    return q, v, d1, beta


def _restore(sysm, snap):
    q, v, d1, beta = snap
    sysm.set_state(q, v)
    sysm.set_frames(d1, beta)


def _timed_steps(sysm, steps, controls, k0, local, graphs=True, clocks=True):
    """Runs `steps` steps (controls(k) applied before step k0 + i) between CUDA
    events with nvidia-smi sampling; returns (ms, per-step iterations, clocks).
    graphs=False: the host drives the Newton rounds."""
    import torch
    sysm.set_graphs(graphs)
    torch.cuda.synchronize()
    clk = Clocks(local) if clocks else None
    if clk:
        clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    its = []
    e0.record()
    for i in range(steps):
        if controls is not None:
            sysm.set_natural_curvature(0, sysm.n_rods, controls(k0 + i))
        sysm.step(1, stats=True)
        its.append(sysm.iterations.copy())
    e1.record()
    torch.cuda.synchronize()
    sysm.set_graphs(True)
    return e0.elapsed_time(e1), np.array(its), clk.stop() if clk else None


def _counts(workload):
    """Per-unit FP64 flops and DRAM bytes by kernel name, counted by ncu on
    this workload: the file's top level for the uneven-rods batch, its
    "workloads" section for the others (none: no counts)."""
    p = os.path.join(ROOT, "profiles", "kernel_fp64_counts.json")
    if not os.path.exists(p):
        return {}, {}
    d = json.load(open(p))
    if workload != "uneven_rods":
        d = d.get("workloads", {}).get(workload, {})
    return dict(d.get("flops_per_unit", {})), dict(d.get("dram_bytes_per_unit", {}))


def _kernel_table(prof, fpu=None, bpu=None, peak_fp64=None):
    """Per kernel: launches, units, time and share; with per-unit counts,
    the achieved FP64 rate against the measured FP64 peak and the DRAM rate
    from the counted bytes."""
    tot = sum(x[2] for x in prof.values()) or 1.0
    out = {k: {"launches": v[0], "units": v[1], "ms_total": round(v[2], 3),
               "share": round(v[2] / tot, 4)} for k, v in prof.items()}
    for k, v in prof.items():
        f = (fpu or {}).get(k)
        if f and v[1] and v[2] > 0 and peak_fp64:
            rate = f * v[1] / (v[2] * 1e-3) / 1e12
            out[k]["fp64_tflops"] = round(rate, 4)
            out[k]["fp64_frac"] = round(rate / (peak_fp64 / 1e3), 4)
        b = (bpu or {}).get(k)
        if b and v[1] and v[2] > 0:
            gbs = b * v[1] / (v[2] * 1e-3) / 1e9
            out[k]["dram_gbs"] = round(gbs, 1)
            out[k]["hbm_frac"] = round(gbs / HBM_PEAK, 4) if HBM_PEAK else None
    return out


def _roofline_fp64(prof, dom, fpu, bpu, peak_fp64):
    """FP64 roofline object of kernel `dom` (achieved = counted flops per
    unit x units / event time), or the latency-bound note without counts."""
    launches, units, kms = prof[dom]
    roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": peak_fp64 / 1e3,
            "peak_source": "measured FP64 FMA throughput (dm_fp64_peak_gflops, this run)",
            "achieved": None, "frac": None, "traffic": None}
    f, b = fpu.get(dom), bpu.get(dom)
    if f and units and kms > 0:
        ach = f * units / launches / (kms / launches * 1e-3) / 1e12
        roof.update({"achieved": ach, "frac": ach / (peak_fp64 / 1e3), "flops_per_unit": f,
                     "unit_name": UNIT_NAME.get(dom), "units_per_launch": units / launches})
        if b:
            roof["traffic"] = b * units / launches
    else:
        roof["note"] = "no per-unit counts for this kernel"
    return roof


def run_other(args):
    """Star robots on the ground, the self-contacting coil, the gripper,
    long rods and the learned warm start: one JSON line each,
    same keys as the headline line; rod-steps/s counts every rod (limb) of
    the batch."""
    import torch
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads
    from paper_2311_18126_gb300 import System, ensure_built, fp64_peak_gflops
    ensure_built()
    peak_fp64 = fp64_peak_gflops()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    if args.workload in ("star_robots", "warm_start"):
        # star robots: seed 3; the warm start deploys on the unseen seed 5
        # and trains on seeds 1000+
        seed = 5 if args.workload == "warm_start" else 3
        desc, params, gait, R_all = shard_of_batch(
            lambda n: workloads.star_robots(n_robots=args.robots * n, seed=seed), ws, rank)
        dt = params["dt"]
        controls = lambda k: workloads.gait_kbar(gait, k * dt)
        line["config"] = {"workload": "star_robots: %d robots of 3-8 limbs x 30 nodes on the "
                          "ground, gait kappabar, dt=5e-3 s, line search" % args.robots,
                          "rods_per_gpu": len(desc["nodes_per_rod"]), "seed": seed,
                          "l2": "no flush: per-iteration working set exceeds L2 at 1024 robots"}
    elif args.workload == "warm_start_rods":
        # the headline batch (seed 2); training batches of seeds 1000+
        desc, params, kbar, R_all = shard_of_batch(
            lambda n: workloads.uneven_rods(n_rods=args.rods * n, seed=2), ws, rank)
        controls = lambda k: kbar
        line["config"] = {"workload": WORKLOAD, "rods_per_gpu": len(desc["nodes_per_rod"]),
                          "l2": "no flush: per-iteration working set (~0.7 GB) exceeds L2"}
    elif args.workload == "long_rods":
        desc, params, kbar, R_all = shard_of_batch(
            lambda n: workloads.uneven_rods(n_rods=64 * n, seed=2, n_min=4000, n_max=6000),
            ws, rank)
        controls = lambda k: kbar
        line["config"] = {"workload": "long_rods: 64 clamped rods of 4000-6000 nodes "
                          "(16k-24k DOFs each), uneven_rods recipe otherwise, dt=1e-3 s; "
                          "rods of >= 2048 DOFs on the partitioned band solve",
                          "rods_per_gpu": 64, "l2": "no flush: working set exceeds L2"}
    elif args.workload == "gripper":
        desc, params, kfn = workloads.gripper()
        R_all = ws * len(desc["nodes_per_rod"])  # one gripper per rank
        dt = params["dt"]
        controls = lambda k: kfn(k * dt)
        line["config"] = {"workload": "gripper: 5 fingers of 60 nodes (L 0.3 m, h 2.5 mm, "
                          "E 0.3 MPa) actuated by random natural curvatures (phibar up to 40 "
                          "deg, ramped over 0.2 s), edge-edge contact with friction mu 0.5 "
                          "between all fingers (one system), dt=1e-3 s, line search",
                          "rods_per_gpu": 5, "l2": "working set in L2 (one system)"}
    else:
        desc, params, _ = workloads.coil(N=500)
        R_all = ws  # one coil per rank
        controls = None
        line["config"] = {"workload": "coil: one 500-node helix collapsing under gravity into "
                          "edge-edge self-contact, dt=2.5e-4 s, line search", "rods_per_gpu": 1,
                          "l2": "working set in L2 (one system)"}
    if args.integrator != "be":
        params = dict(params, integrator=args.integrator)
        line["config"]["integrator"] = args.integrator
    elif args.workload == "long_rods":
        params = dict(params, predictor=args.predictor)
        line["config"]["predictor"] = args.predictor
    R = len(desc["nodes_per_rod"])
    warm = max(args.warmup, 400) if args.workload in ("coil", "gripper") else args.warmup
    line["warmup"] = warm
    if args.workload in ("warm_start", "warm_start_rods"):
        from paper_2311_18126_gb300 import warmstart as wsm
        if args.workload == "warm_start":
            tdesc, tparams, tgait = workloads.star_robots(n_robots=max(args.robots // 4, 64),
                                                          seed=1000 + rank)
            tctl = lambda k: workloads.gait_kbar(tgait, k * dt)
            tsteps, every = 400, 2
            tnote = "%d robots x 400 steps (every 2nd step sampled)" % max(args.robots // 4, 64)
        else:
            tdesc, tparams, tkbar = workloads.uneven_rods(n_rods=1024, seed=1000 + rank)
            tctl = lambda k: tkbar
            tsteps, every = 160, 1
            tnote = "1024 uneven rods of seed 1000 x 160 steps from rest"
        tsys = System(tdesc, tparams)
        feats, tgts = wsm.collect(tsys, tsteps, controls=tctl, every=every)
        tsys.close()
        mlp, norm, losses = wsm.train(feats, tgts, iters=4000, batch=16384, seed=1)
        del feats, tgts
        arms = {}
        variants = [("extrapolation", None, "extrapolate"), ("learned", mlp, "extrapolate")]
        if args.workload == "warm_start_rods":
            # single rods: the length-projected guess, with and without the network
            variants += [("projected", None, "projected"), ("learned_projected", mlp, "projected")]
        for label, model, pred in variants:
            sysm = System(desc, dict(params, predictor=pred))
            sysm.set_natural_curvature(0, R, controls(0))
            tuning = launch_shapes(sysm, args)
            if model is not None:
                sysm.ws_enable()
                sysm.ws_set_model(model, norm)
            for k in range(warm):
                sysm.set_natural_curvature(0, R, controls(k))
                sysm.step(1, stats=False)
            snap = _snapshot(sysm)
            sysm.set_profiling(False)
            ms, its, clocks = _timed_steps(sysm, args.steps, controls, warm, local)
            n_launch = sum(v[0] for v in sysm.get_profile().values())
            ms = max_over_ranks(ms, ws, "cuda")
            _restore(sysm, snap)
            sysm.set_profiling(True)
            _timed_steps(sysm, args.steps, controls, warm, local, clocks=False)
            arms[label] = {"value": job_rate(R_all, args.steps, ms * 1e-3),
                           "ms_per_step": ms / args.steps,
                           "iters_per_rod_step": float(its.mean()),
                           "iters_histogram": np.bincount(its.ravel()).tolist(),
                           "slowest_per_step": float(its.max(1).mean()),
                           "gpu_launches": int(n_launch), "autotune": tuning,
                           "kernels": _kernel_table(sysm.get_profile()), "clocks": clocks}
            sysm.set_profiling(False)
            if model is not None:
                # end to end through the C ABI: pinned host state in and out
                _restore(sysm, snap)
                n = sysm.n_state
                hq = torch.empty(n, dtype=torch.float64, pin_memory=True)
                hv = torch.empty(n, dtype=torch.float64, pin_memory=True)
                hq.numpy()[:], hv.numpy()[:] = snap[0], snap[1]
                e2e_steps = max(3, args.steps // 2)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for i in range(e2e_steps):
                    sysm.set_natural_curvature(0, R, controls(warm + i))
                    sysm.set_state(hq.numpy(), hv.numpy())
                    sysm.step(1, stats=False)
                    sysm.get_state(hq.numpy(), hv.numpy())
                torch.cuda.synchronize()
                te = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
                arms[label]["e2e"] = {"value": job_rate(R_all, e2e_steps, te), "unit": UNIT,
                                      "h2d_bytes_per_step": 2 * n * 8,
                                      "d2h_bytes_per_step": 2 * n * 8,
                                      "note": "setting the state resets the velocity history "
                                              "of the previous-correction features"}
            sysm.close()
        head = "learned_projected" if "learned_projected" in arms else "learned"
        learned = {"speedup_vs_extrapolation": arms[head]["value"] / arms["extrapolation"]["value"],
                   "arm": head, "train_loss": [losses[0], losses[-1]], "arms": arms}
        if "projected" in arms:
            learned["speedup_vs_projected"] = arms[head]["value"] / arms["projected"]["value"]
        line.update({"value": arms[head]["value"],
                     "ms_per_step": arms[head]["ms_per_step"],
                     "learned": learned,
                     "clocks": arms[head]["clocks"],
                     "gpu_launches": arms[head]["gpu_launches"],
                     "e2e": arms[head]["e2e"], "roofline": None,
                     "roofline_note": "solver kernels as in the headline line; the network's "
                                      "tensor-core roofline is the mlp workload's line"})
        line["config"]["training"] = tnote + ", 4000 Adam steps of 16384 segments"
        line["config"]["seed"] = 2 if args.workload == "warm_start_rods" \
            else line["config"].get("seed")
    else:
        sysm = System(desc, params)
        if controls is not None:
            sysm.set_natural_curvature(0, R, controls(0))
        tuning = launch_shapes(sysm, args)
        for k in range(warm):
            if controls is not None:
                sysm.set_natural_curvature(0, R, controls(k))
            sysm.step(1, stats=False)
        snap = _snapshot(sysm)
        sysm.set_profiling(False)
        ms, its, clocks = _timed_steps(sysm, args.steps, controls, warm, local)
        n_launch = sum(v[0] for v in sysm.get_profile().values())
        ms = max_over_ranks(ms, ws, "cuda")
        value = job_rate(R_all, args.steps, ms * 1e-3)
        # the same steps from the same state: host-driven rounds, then profiled
        _restore(sysm, snap)
        host_ms, _, _ = _timed_steps(sysm, args.steps, controls, warm, local, graphs=False,
                                     clocks=False)
        _restore(sysm, snap)
        sysm.set_profiling(True)
        _timed_steps(sysm, args.steps, controls, warm, local, clocks=False)
        prof = sysm.get_profile()
        sysm.set_profiling(False)
        k1 = warm + args.steps
        if args.workload == "long_rods":
            # the same steps from the same state with every rod on the
            # sequential twisted LDL^T
            seq = System(desc, dict(params, long_rod_dofs=-1))
            seq.set_natural_curvature(0, R, controls(0))
            _restore(seq, snap)
            seq_ms, _, _ = _timed_steps(seq, args.steps, controls, warm, local, clocks=False)
            seq.close()
            line["sequential_solve_ms_per_step"] = seq_ms / args.steps
        # end to end through the C ABI: pinned host state in and out every step
        n = sysm.n_state
        hq = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hv = torch.empty(n, dtype=torch.float64, pin_memory=True)
        q0, v0 = sysm.get_state()
        hq.numpy()[:] = q0
        hv.numpy()[:] = v0
        e2e_steps = max(3, args.steps // 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            if controls is not None:
                sysm.set_natural_curvature(0, R, controls(k1 + i))
            sysm.set_state(hq.numpy(), hv.numpy())
            sysm.step(1, stats=False)
            sysm.get_state(hq.numpy(), hv.numpy())
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, ws, "cuda")
        dom = max(prof, key=lambda k: prof[k][2])
        fpu, bpu = _counts(args.workload)
        line.update({"value": value, "ms_per_step": ms / args.steps,
                     "newton": {"iters_mean": float(its.mean()), "iters_max": int(its.max()),
                                "slowest_per_step_mean": float(its.max(1).mean())},
                     "clocks": clocks,
                     "e2e": {"value": job_rate(R_all, e2e_steps, te), "unit": UNIT,
                             "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": 2 * n * 8},
                     "gpu_launches": int(n_launch),
                     "rounds": {"mode": "one CUDA graph per step (device-side while loop "
                                        "over Newton rounds)",
                                "host_loop_ms_per_step": host_ms / args.steps,
                                "note": "host loop timed on the same steps from the same "
                                        "state"},
                     "autotune": tuning,
                     "roofline": _roofline_fp64(prof, dom, fpu, bpu, peak_fp64),
                     "kernels": _kernel_table(prof, fpu, bpu, peak_fp64)})
        if args.workload in ("coil", "gripper"):
            line["contact_pairs"] = sysm.contact_pairs()
        sysm.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def run_calibration(args):
    """Calibration: 64 star robots of 4 limbs on the ground, per-step
    per-limb natural curvatures (kappabar1, kappabar2) as parameters, L2 loss
    on all node positions against a trajectory the solver makes from seeded
    sinusoids, 500 steps with checkpoints every 50.  Times one loss+gradient
    evaluation (forward rollout, re-simulation of each segment, step
    adjoints with the frame chain) and reports rod-steps/s of that pass,
    then takes calibration iterations."""
    import torch
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    import workloads
    from paper_2311_18126_gb300 import System, ensure_built, DismechError
    from paper_2311_18126_gb300.adjoint import rollout, _layout_positions
    ensure_built()
    T, K = 500, 50
    desc, params, gait = workloads.star_robots(n_robots=64, seed=4 + rank, fixed_limbs=4)
    dt = params["dt"]
    R = len(desc["nodes_per_rod"])
    sysm = System(desc, params)
    q0, v0 = sysm.get_state()
    frames = sysm.get_frames()
    nint = gait["nodes_per_limb"] - 2
    spacing = gait["spacing"]
    # per-step per-limb controls c[t, limb, 2] (1/m) -> integrated kappabar per node
    tt = np.arange(T) * dt
    c1 = gait["A"][None, :] * np.sin(2 * np.pi * tt[:, None] / gait["T"][None, :] +
                                     gait["phase"][None, :])
    c_true = np.stack([c1, np.zeros_like(c1)], axis=-1)
    expand = lambda c: (c[:, :, None, :] * spacing).expand(-1, -1, nint, -1).reshape(T, R * nint, 2)
    # every tensor of the pass on the GPU: controls, states, target, loss
    cuda = lambda a: torch.as_tensor(a, dtype=torch.float64).cuda()
    q0t, v0t = cuda(q0), cuda(v0)
    with torch.no_grad():
        target = rollout(sysm, expand(cuda(c_true)), q0t, v0t, frames, K)
    pos = cuda(_layout_positions(np.asarray(desc["nodes_per_rod"])).astype(np.float64))
    c = torch.zeros_like(cuda(c_true), requires_grad=True)

    def loss_grad(cc):
        x = rollout(sysm, expand(cc), q0t, v0t, frames, K)
        loss = (((x - target) ** 2) * pos).sum()
        g, = torch.autograd.grad(loss, [cc])
        return float(loss.detach()), g

    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    t0 = time.perf_counter()
    l0, g = loss_grad(c)
    torch.cuda.synchronize()
    tg = time.perf_counter() - t0
    clocks = clk.stop()
    # calibration iterations with a backtracking step
    losses = [l0]
    step = l0 / float((g * g).sum())
    for _ in range(max(1, args.steps // 10)):
        for _ in range(12):
            trial = (c.detach() - step * g).requires_grad_(True)
            try:
                lt, gt = loss_grad(trial)
            except DismechError:  # a step too long for Newton: shorter
                lt = float("inf")
            if lt < losses[-1]:
                c, g = trial, gt
                losses.append(lt)
                step *= 1.5
                break
            step *= 0.5
    # end to end: the same pass with the controls and their gradient in host
    # memory (the controls go to the device, the gradient comes back)
    c_host = c.detach().cpu().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, g_host = loss_grad(c_host)
    g_host = g_host.numpy()
    te = time.perf_counter() - t0
    line = {"metric": METRIC, "value": R * T / tg, "unit": "rod-steps/s (loss+gradient pass)",
            "n_gpus": ws, "steps": T, "warmup": 0, "ms_per_step": 1e3 * tg / T,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "calibration: 64 star robots x 4 limbs on the ground, "
                       "500 steps, per-step per-limb natural curvature, checkpoints every 50",
                       "rods": R, "params": int(np.prod(c_true.shape)), "seed": 4 + rank},
            "calibration": {"gradient_seconds": tg, "losses": losses}, "clocks": clocks,
            "e2e": {"value": R * T / te, "unit": "rod-steps/s (loss+gradient pass)",
                    "h2d_bytes_per_step": int(R * nint * 2 * 8),
                    "d2h_bytes_per_step": int(c_true.shape[1] * 2 * 8),
                    "note": "the loss+gradient pass with the per-step controls in host memory "
                            "(copied in) and their gradient returned to host memory; the timed "
                            "pass above keeps controls, states, target and gradient on the GPU"},
            "roofline": None}
    if rank == 0:
        print(json.dumps(line))


def run_mlp(args):
    """The warm-start network (4 layers 64 -> 256 -> 256 -> 256 -> 64, BF16
    operands, FP32 accumulation in tensor memory): inference over the
    segments of the 4096-rod headline batch and Adam training steps at the
    training batch size; the tensor-core roofline against the measured BF16
    peak."""
    import torch
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    from paper_2311_18126_gb300 import ensure_built, dismech as dmx
    ensure_built()
    M = args.rows or 444544   # 444456 segments of the 4096-rod batch, padded to 128
    B = 16384             # training batch
    widths = [64, 256, 256, 256, 64]
    fwd = 2 * sum(a * b for a, b in zip(widths[:-1], widths[1:]))  # flops per row
    g = torch.Generator(device="cuda")
    g.manual_seed(1000 + rank)
    X = torch.randn((M, 64), generator=g, device="cuda").to(torch.bfloat16)
    out = torch.empty((M, 64), dtype=torch.float32, device="cuda")
    Yt = torch.randn((B, 4), generator=g, device="cuda")
    mlp = dmx.MLP(61, 4, seed=1)

    def timed(fn, n):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    clk = Clocks(local)
    clk.start()
    # kernel time: back-to-back asynchronous launches between the events,
    # then one check of the error word
    ms_f = timed(lambda: mlp.forward_async(X, out), args.steps)
    mlp.check()
    ms_call = timed(lambda: mlp.forward(X, out), args.steps)
    mlp.set_fused(False)
    ms_layers = timed(lambda: mlp.forward_async(X, out), args.steps)
    mlp.check()
    mlp.set_fused(True)
    ms_t = timed(lambda: mlp.train_step(X[:B], Yt, 1e-4), args.steps)
    clocks = clk.stop()
    ms_f = max_over_ranks(ms_f, ws, "cuda")
    peak = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peak = json.load(open(pk)).get("bf16_tflops")
    src = "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)" if peak else "fallback 1900"
    peak = peak or 1900.0
    ach = fwd * M / (ms_f * 1e-3) / 1e12
    ach_t = 3 * fwd * B / (ms_t * 1e-3) / 1e12
    # end to end: features from pinned host memory in, outputs back
    hX = torch.empty((M, 64), dtype=torch.bfloat16, pin_memory=True)
    hY = torch.empty((M, 64), dtype=torch.float32, pin_memory=True)
    hX.copy_(X)

    def e2e():
        X.copy_(hX, non_blocking=True)
        mlp.forward(X, out)
        hY.copy_(out, non_blocking=True)
    ms_e = timed(e2e, max(3, args.steps // 2))
    line = {"metric": "warm-start network inference, segments/s", "value": ws * M / (ms_f * 1e-3),
            "unit": "segments/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_f, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "mlp: 4 layers 64-256-256-256-64 over %d rows (the segments "
                                   "of the 4096-rod batch); training batch %d" % (M, B),
                       "l2": "inputs and activations (0.9 GB) exceed L2"},
            "clocks": clocks,
            "e2e": {"value": ws * M / (ms_e * 1e-3), "unit": "segments/s",
                    "h2d_bytes_per_step": M * 64 * 2, "d2h_bytes_per_step": M * 64 * 4},
            "gpu_launches": args.steps,
            "roofline": {"bound": "tensor", "kernel": "k_mlp_fused (4 layers, one launch)",
                         "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "peak_source": src, "flops_per_row": fwd, "rows_per_launch": M,
                         "traffic": None,
                         "timing": "CUDA events around back-to-back dm_mlp_forward_async "
                                   "launches",
                         "synchronous_call_ms": ms_call},
            "per_layer_gemms": {"ms": ms_layers,
                                "tflops": fwd * M / (ms_layers * 1e-3) / 1e12,
                                "note": "the same inference as four k_gemm_bf16 launches "
                                        "through global memory"},
            "training": {"ms_per_step": ms_t, "samples_per_s": B / (ms_t * 1e-3),
                         "tflops": ach_t, "frac": ach_t / peak,
                         "note": "forward + backward (data and weight gradients) + Adam"}}
    if rank == 0:
        print(json.dumps(line))
    mlp.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "calibration":
        run_calibration(args)
    elif args.workload == "mlp":
        run_mlp(args)
    elif args.workload != "uneven_rods":
        run_other(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
