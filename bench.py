#!/usr/bin/env python
"""Throughput of the SSP-RK3 / convex-limiting Euler stage on one GB300.

Workload (default): Mach 3 forward-facing step channel [0,3]x[0,1]x[0,0.5],
step x >= 0.6, y <= 0.2, Q1 hexahedra with h = 1/120 (2,242,909 nodes, 27-point
stencil), interior nodes jittered by U[-0.2h, 0.2h] (seed 2007), inflow
rho = 1.4, p = 1, u = (3,0,0), slip walls; FP64 throughout.  One benchmark
step is one SSP-RK3 time step = three euler_steps (Alg. 1 + eq. ssprk3) over
every node; the metric is node-stage updates per second (nodes x 3 stages /
time).  The inputs (matrices and state, ~7 GB) are larger than L2.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank advances its own replica
of the workload (the stage does not shard without a halo exchange, which this
build does not have); value = all ranks' node-stage updates / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D Q1 node-stage updates/s & HBM GB/s: FP64 plain vs FP32-mixed/batched/adjoint"
UNIT = "node-stage updates/s"

# Algorithmic FP64 flops per stored matrix entry (nnz) of each step of Alg. 1
# as counted for the paper's implementation (Table 3; pow and division counted
# by their flops).  Step 5 is the limiter pass, step 6 the final update.
FLOP_PER_NNZ = {"node": 8.0, "edge": 262.0, "diag": 1.0, "low_order": 248.0, "flux_limit": 183.0,
                "limiter_pass": 155.0, "final": 12.0}
# FP64 arithmetic the kernels execute per stored entry: thread-level
# 2 x DFMA + DADD + DMUL from ncu (smsp__sass_thread_inst_executed_op_d*) on
# the step channel at h = 1/80 (17,679,673 entries), first euler_step after
# three warm-up steps.  This is the `achieved`
# work of the FP64 roofline; the paper's per-step counts above overstate what
# these kernels execute (lambda_max once per unordered edge, flux differences
# once per pair, powers without pow, tests on 32-bit words), so a rate from
# them can exceed the pipe.
FP64_FLOP_PER_NNZ_EXECUTED = {"node": 3.5, "edge": 45.3, "diag": 11.2, "low_order": 51.0, "flux_limit": 44.0,
                              "limiter_pass": 14.6, "final": 10.6}
# FP64 pipe busy fraction (sm__pipe_fp64_cycles_active, % of active cycles) of
# the same capture: the pipe also issues compares, conversions and min/max.
FP64_PIPE_BUSY_NCU = {"node": 0.855, "edge": 0.854, "diag": 0.701, "low_order": 0.891, "flux_limit": 0.875,
                      "limiter_pass": 0.821, "final": 0.848}
# FP64 peak from the unit counts and the maximum SM clock: 152 SMs x 2 FP64
# FMA/clk x 2 flop x 2.070 GHz (nominal 1.25 TFLOP/s).  The roofline uses the
# rate the library's own FMA-stream probe measures in the same run
# (idp_probe_fp64_peak); this figure is its fallback.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum,
# one pass, no replay) on the workloads of this file at full size: the step
# channel at h = 1/120 (FP64) and the 128^3 Sod cube (FP32-mixed), one stage
# after three warm-up steps (profiles/ holds the launch lists).
NCU_TRAFFIC_BYTES = {"node": 0.225e9, "edge": 4.843e9, "diag": 4.018e9, "low_order": 4.073e9,
                     "flux_limit": 4.122e9, "limiter_pass": 6.944e9, "final": 3.210e9}
NCU_TRAFFIC_BYTES_MIXED = {"node": 0.138e9, "edge": 1.729e9, "low_order": 2.198e9, "flux_limit": 1.820e9,
                           "limiter_pass": 3.617e9, "final": 1.608e9}


# The byte and flop model of the method per stored entry and stage (3D Q1,
# FP64): B_sched, the canonical five-sweep schedule with P_ij recomputed
# (170 B per entry; 140 B with FP32 d and l), B_min, every matrix read once and
# the state in and out (1,060 B per node-stage at 27 entries per row), and the
# paper's operation count of ~869 flop per entry and stage (Table 3).
B_SCHED_PER_ENTRY = {"fp64": 170.0, "fp32_mixed": 140.0}
B_MIN_PER_NODE_STAGE = 1060.0
F_PAPER_PER_ENTRY = 869.0


def byte_model(rate, nodes, nnz, ncu_bytes_per_stage, hbm_peak_gbs, fp_peak_tflops, exec_flop_per_entry, precision):
    """Measured DRAM bytes per node-stage against B_sched and B_min, and the
    bound-implied fraction: the achieved node-stage rate over the smaller of
    the HBM ceiling (peak / B_sched) and the FP ceiling (peak / flops per
    node-stage), with the paper's flop count and with the kernels' executed
    one (ncu)."""
    per_node = nnz / nodes
    b_sched = B_SCHED_PER_ENTRY[precision] * per_node
    hbm_ceiling = hbm_peak_gbs * 1e9 / b_sched
    out = {"entries_per_node": per_node, "b_sched_per_node_stage": b_sched,
           "b_min_per_node_stage": B_MIN_PER_NODE_STAGE,
           "ncu_dram_bytes_per_node_stage": None if ncu_bytes_per_stage is None else ncu_bytes_per_stage / nodes,
           "hbm_ceiling": hbm_ceiling}
    if ncu_bytes_per_stage is not None:
        out["ncu_bytes_over_b_sched"] = ncu_bytes_per_stage / nodes / b_sched
    if fp_peak_tflops:
        fp_paper = fp_peak_tflops * 1e12 / (F_PAPER_PER_ENTRY * per_node)
        out["fp_ceiling_paper_flops"] = fp_paper
        out["bound_implied_frac_paper_flops"] = rate / min(hbm_ceiling, fp_paper)
        if exec_flop_per_entry:
            fp_exec = fp_peak_tflops * 1e12 / (exec_flop_per_entry * per_node)
            out["fp_ceiling_executed_flops"] = fp_exec
            out["bound_implied_frac_executed_flops"] = rate / min(hbm_ceiling, fp_exec)
    else:
        out["bound_implied_frac"] = rate / hbm_ceiling
    return out


# Algorithmic bytes of the FP32-mixed kernels (each array the kernel must read
# or write once; neighbour gathers counted once per node): bytes per stored
# entry (slot) and per node.
MIXED_BYTES = {"node": (0, 92), "edge": (35, 52), "low_order": (32, 164),
               "flux_limit": (36, 116), "limiter_pass": (60, 112), "final": (36, 124)}
# The same with row patterns (structured grids): the column index (4 B),
# transpose map (4 B), flags (1 B) and table code (2 B) of a slot come from
# the row's pattern (a 2-byte id per node and a table that stays on chip);
# Step 3 keeps the column stream.
MIXED_BYTES_PATTERNS = {"node": (0, 92), "edge": (28, 54), "low_order": (32, 164),
                        "flux_limit": (30, 118), "limiter_pass": (52, 114), "final": (28, 126)}


def _hbm_peak():
    """Measured copy bandwidth of this machine (GB/s), else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


_PEAK64 = {}


def fp64_peak(stream, bus_id=None):
    """Measured FP64 FMA rate of this GPU (idp_probe_fp64_peak, best of three
    launches) with the SM clocks sampled while it runs; falls back to the
    unit-count figure if the probe fails.  Measured once per process."""
    if "v" not in _PEAK64:
        _PEAK64["v"] = _measure_fp64_peak(stream, bus_id)
    return _PEAK64["v"]


def _measure_fp64_peak(stream, bus_id):
    from paper_2007_00094_gb300.idp import IdpError, idp_probe_fp64_peak

    sampler = ClockSampler(bus_id=bus_id)
    sampler.start()
    try:
        best = 0.0
        for _ in range(3):
            best = max(best, idp_probe_fp64_peak(1 << 20, stream)[0])
    except IdpError:
        best = None
    clocks = sampler.stop()
    if best is None:
        return FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (probe failed)", clocks
    mhz = clocks["sm_mhz"] if clocks else None
    return best, (f"measured: FP64 FMA stream of libidp (idp_probe_fp64_peak), best of 3 launches, "
                  f"median SM clock {mhz} MHz"), clocks


def _time_steps(solver, stream, steps, warmup, profile=True):
    """Warm-up, then steps SSP-RK3 steps timed with CUDA events; returns
    (ms per step, per-kernel profile or None)."""
    import torch

    solver.step(warmup)
    solver.synchronize()
    if profile:
        solver.profile(True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    solver.synchronize()
    prof = None
    if profile:
        prof = solver.profile_read()
        solver.profile(False)
    return e0.elapsed_time(e1) / steps, prof


def pattern_batched(stream, args):
    """256 independent Riemann problems on slip-walled cubes of random size,
    advanced together (per-instance tau_n); schedule chosen by the autotuner."""
    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver

    parts = W.random_riemann_batch(n_instances=args.batch_instances, side_range=(8, 48), seed=4)
    mesh, off, U0 = W.concat_meshes([m for m, _ in parts], [u for _, u in parts])
    del parts
    out = {"config": {"workload": f"{args.batch_instances}_riemann_cubes_sides_8-48_seed4", "nodes": mesh.n_nodes,
                      "instances": args.batch_instances, "steps_timed": args.pattern_steps, "warmup": args.warmup}}
    for name, prec in (("fp64", 0), ("fp32_mixed", 1)):
        s = Solver(mesh, stream=stream, precision=prec)
        s.set_instances(off)
        s.init_state(U0)
        block, graph, persistent, ms_tuned = s.autotune(steps=1)
        ms, _ = _time_steps(s, stream, args.pattern_steps, args.warmup, profile=False)
        out[name] = {"value": mesh.n_nodes * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "schedule": {"block": block, "cuda_graph": graph, "persistent": persistent,
                                  "autotune_ms_per_step": ms_tuned},
                     "gpu_launches_per_step": 3 if persistent else (21 if prec == 0 else 18)}
        # every schedule on the same batch, for the record
        sched = {}
        for pers in (False, True):
            for g in (False, True):
                s.set_schedule(block, g, pers)
                s.init_state(U0)
                sched[f"{'persistent' if pers else 'per_step'}_{'graph' if g else 'stream'}"] = \
                    _time_steps(s, stream, 2, 3, profile=False)[0]
        out[name]["ms_per_step_by_schedule_at_block"] = sched
        # per-kernel times (per-step kernels at the chosen block size) and per stored entry
        s.set_schedule(block, False, False)
        s.init_state(U0)
        _, prof = _time_steps(s, stream, 2, 3, profile=True)
        out[name]["kernels_ms_per_launch"] = {k: v[0] / v[1] for k, v in prof.items() if v[1]}
        out[name]["kernels_ns_per_entry"] = {k: v[0] / v[1] * 1e6 / s.nnz for k, v in prof.items() if v[1]}
        out["config"]["nnz"] = s.nnz
        s.close()
    out["config"]["boundary_node_fraction"] = float((mesh.bc != 0).mean())
    return out


def pattern_mixed(stream, args):
    """FP32-mixed vs FP64 on the 3D Sod tube, 128^3 nodes, slip walls."""
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver

    mesh = W.sod_cube_mesh(args.sod_n)
    U0 = W.sod_state(mesh)
    out = {"config": {"workload": f"sod_tube_{args.sod_n}^3_slip_walls", "nodes": mesh.n_nodes,
                      "steps_timed": args.pattern_steps, "warmup": args.warmup,
                      "accuracy_steps": max(args.sod_steps, args.pattern_steps + args.warmup)}}
    states, times, bounds = {}, {}, {}
    for name, prec in (("fp64", 0), ("fp32_mixed", 1)):
        s = Solver(mesh, stream=stream, precision=prec)
        s.init_state(U0)
        ms, prof = _time_steps(s, stream, args.pattern_steps, args.warmup)
        # untimed: continue to the accuracy horizon
        s.step(max(args.sod_steps - args.pattern_steps - args.warmup, 0))
        s.synchronize()
        states[name] = s.get_state()
        times[name] = s.time()[0]
        st, rep = s.check_bounds()
        bounds[name] = {"status": st, "rho_min": rep.rho_min, "eps_min": rep.eps_min}
        entry = {"value": mesh.n_nodes * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                 "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in prof.items() if v[1]}}
        if prec == 1:
            entry["entry_table_values"] = s.entry_table_size()
            entry["row_patterns"] = s.row_pattern_count()
            dom = max(prof, key=lambda k: prof[k][0])
            dom_ms, dom_n = prof[dom]
            per_slot, per_node = (MIXED_BYTES_PATTERNS if entry["row_patterns"] else MIXED_BYTES)[dom]
            bytes_per_launch = per_slot * s.nnz + per_node * mesh.n_nodes
            peak, src = _hbm_peak()
            achieved = bytes_per_launch / (dom_ms / dom_n * 1e-3) / 1e9
            traffic = NCU_TRAFFIC_BYTES_MIXED.get(dom) if args.sod_n == 128 else None
            entry["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                                 "work": f"{per_slot} B/entry x {s.nnz} + {per_node} B/node x {mesh.n_nodes}"}
            stage_bytes = sum(NCU_TRAFFIC_BYTES_MIXED.values()) if args.sod_n == 128 else None
            entry["byte_model"] = byte_model(entry["value"], mesh.n_nodes, s.nnz, stage_bytes, peak, None, None,
                                             "fp32_mixed")
        out[name] = entry
        s.close()
    # the same mixed stage reading per-entry FP32 arrays instead of the entry table
    s = Solver(mesh, stream=stream, precision=1, entry_table=0)
    s.init_state(U0)
    ms_pe, prof_pe = _time_steps(s, stream, args.pattern_steps, args.warmup)
    s.close()
    out["fp32_mixed"]["per_entry_arrays"] = {
        "ms_per_step": ms_pe, "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in prof_pe.items() if v[1]}}
    ref = states["fp64"]
    scale = np.abs(ref).max(axis=1)
    scale = np.where(scale > 1e-12 * scale.max(), scale, scale.max())
    err = np.abs(states["fp32_mixed"] - ref).mean(axis=1) / scale
    out["fp32_mixed"]["l1_error_vs_fp64"] = {f: float(e) for f, e in zip(["rho", "m_x", "m_y", "m_z", "E"], err)}
    out["fp32_mixed"]["accuracy_time"] = {"fp64": times["fp64"], "fp32_mixed": times["fp32_mixed"]}
    out["fp32_mixed"]["invariants"] = bounds
    out["fp32_mixed"]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp32_mixed"]["ms_per_step"]
    return out


def pattern_adjoint(stream, args):
    """Gradient of J = sum_{x_i in [0.4,0.6]^3} m_i p_i(U^N) with respect to U^0
    through N FP64 SSP-RK3 steps on the 64^3 periodic vortex with eight
    Gaussian density bumps, checkpoints every 10 steps: cost of the recorded
    forward run and of the reverse sweep against a plain forward run, and a
    central-difference check along random directions."""
    import numpy as np
    import torch

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver
    from paper_2007_00094_gb300.objectives import BoxPressure

    mesh = W.vortex_mesh(args.adj_n)
    U0 = W.bumpy_vortex_state(mesh)
    N, every = args.adj_steps, 10
    s = Solver(mesh, stream=stream)
    J = BoxPressure(mesh.x, s.matrices()[4])

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    s.init_state(U0)
    s.step(args.warmup)
    s.synchronize()
    s.init_state(U0)
    fwd_ms, _ = timed(lambda: s.step(N))
    s.synchronize()
    s.init_state(U0)
    rec_ms, _ = timed(lambda: s.adjoint_record(N, every))
    seed = torch.as_tensor(J.gradient(s.get_state()), device="cuda")
    s.profile(True)
    bwd_ms, g = timed(lambda: s.adjoint_backward(seed))
    prof = s.profile_read()
    s.profile(False)
    g = g.cpu().numpy()

    def run(V):
        s.init_state(V)
        s.step(N)
        return J(s.get_state())

    # central differences of the forward run; the map is piecewise smooth,
    # so the agreement is limited by the branch points a difference crosses
    rng = np.random.default_rng(16)
    fd_err = {1e-6: [], 1e-8: []}
    for _ in range(args.adj_fd_directions):
        v = rng.standard_normal(U0.shape) * np.abs(U0)
        ad = float((g * v).sum())
        for eps in fd_err:
            fd = (run(U0 + eps * v) - run(U0 - eps * v)) / (2 * eps)
            fd_err[eps].append(abs(fd - ad) / abs(ad))
    s.close()
    node_stages = mesh.n_nodes * 3 * N
    adj = {k: v for k, v in prof.items() if k.startswith("adj_") and v[1]}
    return {"config": {"workload": f"bumpy_vortex_{args.adj_n}^3_periodic_8_bumps_seed5", "nodes": mesh.n_nodes,
                       "steps": N, "checkpoint_every": every,
                       "functional": "sum over x_i in [0.4,0.6]^3 of m_i p_i(U^N)", "box_nodes": J.n_inside},
            "value": node_stages / ((rec_ms + bwd_ms) * 1e-3), "unit": "node-stage gradient updates/s",
            "forward_ms": fwd_ms, "record_ms": rec_ms, "backward_ms": bwd_ms,
            "backward_over_forward": bwd_ms / fwd_ms, "gradient_over_forward": (rec_ms + bwd_ms) / fwd_ms,
            "reverse_kernels_ms_per_launch": {k: v[0] / v[1] for k, v in adj.items()},
            "backward_share_forward_recompute": sum(v[0] for k, v in prof.items() if not k.startswith("adj_"))
            / sum(v[0] for v in prof.values()),
            "fd_check": {"directions": args.adj_fd_directions,
                         "max_rel_err": {f"{e:.0e}": (max(v) if v else None) for e, v in fd_err.items()}}}


def pattern_adjoint_fd(stream, args):
    """Where the finite differences of the differentiation workload lose
    against its derivative: central differences of J(U^N) along the seeded
    directions for a range of eps against the CUDA adjoint's <dJ/dU^0, v>,
    and, for the first args.adj_fd_trace_steps SSP-RK3 steps, the number of
    limiter values whose branch (t = 0, 0 < t < 1, t = 1) differs between the
    +eps and the -eps run (stages run one at a time with their traces, the
    RK blend on the host)."""
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver
    from paper_2007_00094_gb300.objectives import BoxPressure

    mesh = W.vortex_mesh(args.adj_n)
    U0 = W.bumpy_vortex_state(mesh)
    N = args.adj_steps
    s = Solver(mesh, stream=stream)
    J = BoxPressure(mesh.x, s.matrices()[4])
    s.init_state(U0)
    s.adjoint_record(N, 10)
    g = s.adjoint_backward(J.gradient(s.get_state()))
    dirs = W.perturbation_directions(U0, args.adj_fd_directions, seed=16)

    def run(V):
        s.init_state(V)
        s.step(N)
        return J(s.get_state())

    def branch(l):
        return np.digitize(l, [1e-300, 1.0]).astype(np.uint8)

    def classes(V, steps):
        out = []
        U = V
        for _ in range(steps):
            s.init_state(U)
            tau = s.euler_step(trace=True)
            out.append([branch(s.field("l4")), branch(s.field("l5"))])
            E1 = s.get_state()
            s.euler_step(tau=tau, trace=True)
            out.append([branch(s.field("l4")), branch(s.field("l5"))])
            U2 = 0.75 * U + 0.25 * s.get_state()
            s.init_state(U2)
            s.euler_step(tau=tau, trace=True)
            out.append([branch(s.field("l4")), branch(s.field("l5"))])
            U = 1.0 / 3.0 * U + 2.0 / 3.0 * s.get_state()
            del E1
        return out

    eps_list = [1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10]
    rows = []
    for k, v in enumerate(dirs):
        ad = float((g * v).sum())
        row = {"adjoint": ad, "fd_rel_err": {}, "limiter_branch_changes_first_steps": {}}
        for eps in eps_list:
            fd = (run(U0 + eps * v) - run(U0 - eps * v)) / (2 * eps)
            row["fd_rel_err"][f"{eps:.0e}"] = abs(fd - ad) / abs(ad)
        if k == 0:
            for eps in (1e-6, 1e-8):
                cp = classes(U0 + eps * v, args.adj_fd_trace_steps)
                cm = classes(U0 - eps * v, args.adj_fd_trace_steps)
                row["limiter_branch_changes_first_steps"][f"{eps:.0e}"] = [
                    int(sum((a != b).sum() for a, b in zip(x, y))) for x, y in zip(cp, cm)]
        rows.append(row)
    s.close()
    return {"config": {"workload": f"bumpy_vortex_{args.adj_n}^3_periodic_8_bumps_seed5", "steps": N,
                       "directions_seed": 16, "traced_steps": args.adj_fd_trace_steps,
                       "entries": int(mesh.n_nodes * 27)},
            "directions": rows}


def pattern_relaxation(stream, args):
    """Accuracy of the bound relaxation (idp_config.relax): L1 density error
    of the isentropic vortex against its exact translation at t >= 0.05 on
    periodic n x n x 3 meshes, FP64, with and without relaxation, and the
    observed orders."""
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver

    out = {"config": {"workload": "isentropic_vortex_periodic_n_x_n_x_3_t0.05", "n": [40, 80, 160]}}
    for relax in (0, 1):
        errs = []
        for n in out["config"]["n"]:
            mesh = W.box_mesh((n, n, 3), periodic=(True, True, True))
            s = Solver(mesh, stream=stream, relax=relax)
            s.init_state(W.vortex_state(mesh))
            while s.time()[0] < 0.05:
                s.step(1)
            t = s.time()[0]
            errs.append(float(np.abs(s.get_state()[0] - W.vortex_state(mesh, t=t)[0]).mean()))
            s.close()
        out["relaxed" if relax else "plain"] = {
            "l1_density_error": errs, "orders": [float(np.log2(errs[k] / errs[k + 1])) for k in range(len(errs) - 1)]}
    return out


def pattern_q1_2d(stream, args):
    """2D Q1 variant (quadrilaterals, 9-point stencil): the Mach 3 forward-facing
    step [0,3]x[0,1] with h = 1/m2d, jittered interior, FP64 and FP32-mixed."""
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver

    mesh = W.forward_step_mesh_2d(m=args.m2d, jitter=0.2, seed=2007)
    U0 = W.forward_step_state(mesh)
    out = {"config": {"workload": f"mach3_forward_facing_step_2d_h1/{args.m2d}_jitter0.2_seed2007",
                      "nodes": mesh.n_nodes, "stencil": "Q1 9-point", "steps_timed": args.pattern_steps,
                      "warmup": args.warmup}}
    peak_hbm, src = _hbm_peak()
    for name, prec in (("fp64", 0), ("fp32_mixed", 1)):
        s = Solver(mesh, stream=stream, precision=prec)
        s.init_state(U0)
        ms, prof = _time_steps(s, stream, args.pattern_steps, args.warmup)
        out["config"]["nnz"] = s.nnz
        dom = max(prof, key=lambda k: prof[k][0])
        dom_ms, dom_n = prof[dom]
        per_launch_s = dom_ms / dom_n * 1e-3
        if prec == 0:
            achieved = FP64_FLOP_PER_NNZ_EXECUTED[dom] * s.nnz / per_launch_s / 1e12
            peak64, peak64_src, _ = fp64_peak(stream)
            roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                    "frac": achieved / peak64, "traffic": None, "peak_source": peak64_src,
                    "work": f"{FP64_FLOP_PER_NNZ_EXECUTED[dom]} executed FP64 flop/nnz (ncu, 3D step channel) x "
                            f"{s.nnz} nnz per launch"}
        else:
            per_slot, per_node = (MIXED_BYTES_PATTERNS if s.row_pattern_count() else MIXED_BYTES)[dom]
            achieved = (per_slot * s.nnz + per_node * mesh.n_nodes) / per_launch_s / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                    "frac": achieved / peak_hbm, "traffic": None, "peak_source": src,
                    "work": f"{per_slot} B/entry x {s.nnz} + {per_node} B/node x {mesh.n_nodes}"}
        U = s.get_state()
        st, rep = s.check_bounds()
        out[name] = {"value": mesh.n_nodes * 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
                     "roofline": roof, "m_z_max_abs": float(np.abs(U[3]).max()),
                     "invariants": {"status": st, "rho_min": rep.rho_min, "eps_min": rep.eps_min}}
        s.close()
    out["fp32_mixed"]["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["fp32_mixed"]["ms_per_step"]
    return out


def pattern_renumber(stream, args):
    """Row order: the step channel (h = 1/m) with its nodes in the generator's
    lexicographic order, randomly shuffled (seeded) as given, and shuffled but
    renumbered by the library (idp_config.renumber: 1 reverse Cuthill-McKee,
    2 Morton order of the node coordinates, also from the lexicographic
    order); FP64 and FP32-mixed ms per SSP-RK3 step."""
    import numpy as np

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import Solver

    mesh = W.forward_step_mesh(m=args.m, jitter=0.2, seed=2007)
    U0 = W.forward_step_state(mesh)
    rng = np.random.default_rng(11)
    p = rng.permutation(mesh.n_nodes)
    inv = np.empty_like(p)
    inv[p] = np.arange(mesh.n_nodes)
    shuf = W.HexMesh(x=mesh.x[inv], cells=p[mesh.cells], cell_xyz=mesh.cell_xyz, bc=mesh.bc[inv], volume=mesh.volume,
                     inflow=mesh.inflow, name="shuffled")
    U_shuf = U0[:, inv]
    out = {"config": {"workload": f"mach3_forward_facing_step_h1/{args.m}_nodes_shuffled_seed11", "nodes": mesh.n_nodes,
                      "steps_timed": args.pattern_steps, "warmup": args.warmup}}
    for name, prec in (("fp64", 0), ("fp32_mixed", 1)):
        row = {}
        for label, m, u, ren in (("lexicographic", mesh, U0, 0), ("shuffled", shuf, U_shuf, 0),
                                 ("shuffled_renumbered", shuf, U_shuf, 1), ("shuffled_morton", shuf, U_shuf, 2),
                                 ("lexicographic_morton", mesh, U0, 2)):
            s = Solver(m, stream=stream, precision=prec, renumber=ren)
            s.init_state(u)
            row[label] = _time_steps(s, stream, args.pattern_steps, args.warmup, profile=False)[0]
            s.close()
        out[name] = {"ms_per_step": row}
    return out


def pattern_sharded(stream, args):
    """The sharded stage on one GPU (idp_shards_*, Sec. 4.1, Fig. 1-2): the
    step channel's rows in 2 and 4 contiguous ranges with one ghost layer,
    halo exchanges (gather kernel, device copy, scatter kernel) between the
    stage's phases.  FP64 and FP32-mixed ms per SSP-RK3 step against the
    unsharded stage on the same matrices, the bytes exchanged per step, and
    whether the states after the timed steps are bitwise equal."""
    import numpy as np
    import torch

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import ShardedSolver, Solver

    mesh = W.forward_step_mesh(m=args.m, jitter=0.2, seed=2007)
    U0 = W.forward_step_state(mesh)
    s = Solver(mesh, stream=stream)
    rowptr, col, mij, cij, mi = s.matrices()
    s.close()
    sp = dict(rowptr=rowptr, col=col, mij=mij, cij=cij, mi=mi, bc=mesh.bc, inflow=mesh.inflow)
    steps, warm = args.pattern_steps, args.warmup

    def timed(solver):
        solver.init_state(U0)
        solver.step(warm)
        solver.synchronize()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(steps)
        e1.record(stream)
        solver.synchronize()
        return e0.elapsed_time(e1) / steps, solver.get_state()

    out = {"config": {"workload": f"mach3_forward_facing_step_h1/{args.m}_jitter0.2_seed2007", "nodes": mesh.n_nodes,
                      "nnz": len(col), "steps_timed": steps, "warmup": warm}}
    for name, prec in (("fp64", 0), ("fp32_mixed", 1)):
        ref = Solver(sparsity=sp, stream=stream, precision=prec)
        ms_ref, U_ref = timed(ref)
        ref.close()
        row = {"unsharded_ms_per_step": ms_ref}
        for k in (2, 4):
            sh = ShardedSolver(sp, n_shards=k, stream=stream, precision=prec)
            ms, U = timed(sh)
            nn, ne, launches = sh.halo_size()
            ghosts = sum(sh.plan.info(q)[0] - (sh.plan.info(q)[2] - sh.plan.info(q)[1]) for q in range(k))
            sh.close()
            # per stage: alpha (1 field), R (5), U (5) at ghost nodes, l twice at halo entries;
            # alpha, R and l are FP32 in the mixed stage
            w = 8 if prec == 0 else 4
            nbytes = 3 * (w * 6 * nn + 8 * 5 * nn + w * 2 * ne)
            row[f"shards_{k}"] = {"ms_per_step": ms, "over_unsharded": ms / ms_ref,
                                  "value": mesh.n_nodes * 3 / (ms * 1e-3), "unit": "node-stage updates/s",
                                  "ghost_nodes": int(ghosts), "halo_node_values_per_field": nn,
                                  "halo_entry_values": ne, "exchanged_bytes_per_step": nbytes,
                                  "launches_per_step": launches / steps,
                                  "bitwise_equal_to_unsharded": bool(np.array_equal(U, U_ref))}
        out[name] = row
    return out


def pattern_steps(stream, args):
    """A plain run for profilers: `--warmup` SSP-RK3 steps, then `--steps`
    more, of one workload (`--case channel`: the step channel h = 1/m;
    `--case sod`: the Sod cube with --sod-n nodes per axis) in one precision
    (`--precision`), unsharded or in `--shards` shards; prints ms per step."""
    import torch

    from paper_2007_00094_gb300 import workloads as W
    from paper_2007_00094_gb300.idp import ShardedSolver, Solver

    if args.case == "sod":
        mesh = W.sod_cube_mesh(args.sod_n)
        U0 = W.sod_state(mesh)
    else:
        mesh = W.forward_step_mesh(m=args.m, jitter=0.2, seed=2007)
        U0 = W.forward_step_state(mesh)
    if args.shards > 1:
        s = Solver(mesh, stream=stream)
        rowptr, col, mij, cij, mi = s.matrices()
        s.close()
        sp = dict(rowptr=rowptr, col=col, mij=mij, cij=cij, mi=mi, bc=mesh.bc, inflow=mesh.inflow)
        solver = ShardedSolver(sp, n_shards=args.shards, stream=stream, precision=args.precision)
    else:
        solver = Solver(mesh, stream=stream, precision=args.precision)
    solver.init_state(U0)
    solver.step(args.warmup)
    solver.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    solver.synchronize()
    solver.close()
    return {"case": args.case, "nodes": mesh.n_nodes, "precision": args.precision, "shards": args.shards,
            "warmup": args.warmup, "steps": args.steps, "ms_per_step": e0.elapsed_time(e1) / args.steps}


def job_rate(local_ms, units_per_rank, dist=None, device="cpu"):
    """Whole-job rate of a weak-scaling run: the slowest rank's time (max over
    ranks) and all ranks' units divided by it.  Returns (ms_max, units/s)."""
    import torch

    ws = dist.get_world_size() if dist is not None else 1
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, ws * units_per_rank / (ms_max * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ["pci.bus_id", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv"), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(", ") for r in self.out.read().strip().splitlines() if r.strip()]
        self.out.close()
        if self.bus_id:
            mine = [r for r in rows if r and r[0].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < len(self.FIELDS):
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for q, name in enumerate(names):
                if r[5 + q].strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_mesh(mesh):
    """The oracle's own assembly of a workloads mesh, and its wall time."""
    import oracle as O

    O.build()
    t0 = time.perf_counter()
    om = O.assemble(mesh)
    return om, time.perf_counter() - t0


def _oracle_rate(om, U, n_threads, seconds_budget, max_stages):
    """euler_steps of the oracle from U until about seconds_budget (at least
    one): node-stage updates/s and the stages run."""
    import oracle as O

    prm = O.default_params(n_threads=n_threads)
    stages, elapsed, V = 0, 0.0, U
    while stages < 1 or (elapsed < seconds_budget and stages < max_stages):
        t0 = time.perf_counter()
        V, tau, st, _ = O.euler_step(om, V, params=prm)
        elapsed += time.perf_counter() - t0
        stages += 1
        if st != 0:
            break
    return om.n * stages / elapsed, stages, elapsed


def cpu_baseline(mesh, U, seconds_budget=15.0):
    """The FP64 oracle, as it stands, on the host cores, on the benchmark's own
    channel mesh (assembled by the oracle, untimed): OpenMP over rows on all
    cores for about seconds_budget, and single-threaded for one euler_step
    (results are bitwise the same; the j-loop order does not change).  Also the
    17^3 periodic vortex run in full (20 SSP-RK3 steps) in both modes."""
    import oracle as O
    from paper_2007_00094_gb300 import workloads as W

    cores = os.cpu_count() or 1
    om, t_asm = _oracle_mesh(mesh)
    v_omp, n_omp, s_omp = _oracle_rate(om, U, cores, seconds_budget, 200)
    v_one, n_one, s_one = _oracle_rate(om, U, 1, 0.0, 1)
    del om
    vm = W.vortex_mesh(17)
    vom, _ = _oracle_mesh(vm)
    c1 = {}
    for label, nt in (("openmp", cores), ("single_thread", 1)):
        t0 = time.perf_counter()
        O.run(vom, W.vortex_state(vm), 20, O.default_params(n_threads=nt))
        dt = time.perf_counter() - t0
        c1[label] = {"value": vm.n_nodes * 3 * 20 / dt, "seconds": dt, "threads": nt}
    return {"value": v_omp, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_omp} euler_steps of the FP64 oracle on the benchmark mesh itself ({mesh.n_nodes} nodes), "
                      f"{s_omp:.1f} s on {cores} threads; oracle assembly {t_asm:.1f} s untimed",
            "modes": {"openmp": {"value": v_omp, "threads": cores, "stages": n_omp, "seconds": s_omp},
                      "single_thread": {"value": v_one, "threads": 1, "stages": n_one, "seconds": s_one}},
            "vortex_17^3_20_steps_in_full": c1}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on all host cores
    (OpenMP over rows), on the benchmark's own channel mesh; each step is one
    SSP-RK3 step (three euler_steps) over every node, as in the GPU arm."""
    import oracle as O
    from paper_2007_00094_gb300 import workloads as W

    mesh = W.forward_step_mesh(m=args.m, jitter=0.2, seed=2007)
    om, _ = _oracle_mesh(mesh)
    V = W.forward_step_state(mesh)
    cores = os.cpu_count() or 1
    prm = O.default_params(n_threads=cores)
    for _ in range(args.warmup):
        V, _, _ = O.ssprk3_step(om, V, prm)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        V, _, st = O.ssprk3_step(om, V, prm)
    dt = time.perf_counter() - t0
    value = mesh.n_nodes * 3 * args.steps / dt
    sample = (f"each step = one SSP-RK3 step (3 euler_steps) of the FP64 oracle on the benchmark mesh itself "
              f"({mesh.n_nodes} nodes, {om.nnz} entries), {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args.m, mesh.n_nodes, om.nnz, args),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _channel_nodes(m):
    nz = m // 2 + 1
    return (3 * m + 1) * (m + 1) * nz - (3 * m - (6 * m) // 10) * ((2 * m) // 10) * nz


def _config(m, nodes, nnz, args):
    return {"workload": f"mach3_forward_facing_step_h1/{m}_jitter0.2_seed2007", "nodes": nodes,
            "nnz": nnz, "stencil": "Q1 27-point", "step": "one SSP-RK3 step = 3 euler_steps",
            "limiter_passes": 2, "newton_steps": 2, "cfl": 0.5,
            "l2": "inputs larger than L2 (matrices and state resident in HBM, ~7 GB)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=120, help="cells per unit length of the channel mesh")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-patterns", action="store_true", help="skip the FP32-mixed / batched / adjoint lines")
    ap.add_argument("--pattern-steps", type=int, default=5)
    ap.add_argument("--sod-n", type=int, default=128)
    ap.add_argument("--sod-steps", type=int, default=100,
                    help="total steps (timed ones included) after which the mixed path is compared with FP64")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--adj-n", type=int, default=64, help="nodes per axis of the adjoint workload")
    ap.add_argument("--adj-steps", type=int, default=100)
    ap.add_argument("--adj-fd-directions", type=int, default=2)
    ap.add_argument("--adj-fd-trace-steps", type=int, default=10)
    ap.add_argument("--m2d", type=int, default=1000, help="cells per unit length of the 2D channel mesh")
    ap.add_argument("--case", default="channel", choices=["channel", "sod"], help="workload of --only steps")
    ap.add_argument("--precision", type=int, default=0, help="0 FP64, 1 FP32-mixed (--only steps)")
    ap.add_argument("--shards", type=int, default=1, help="shards on one GPU (--only steps)")
    ap.add_argument("--only", choices=["fp32_mixed", "batched", "adjoint", "adjoint_fd", "relaxation", "q1_2d",
                                       "renumber", "sharded", "steps"],
                    help="run one pattern alone and print its JSON (no headline line)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")

    ws, rank, local = _dist()
    from paper_2007_00094_gb300 import workloads as W

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    from paper_2007_00094_gb300 import build
    from paper_2007_00094_gb300.idp import Solver

    torch.cuda.set_device(local)
    if args.only:
        build.build()
        run = {"fp32_mixed": pattern_mixed, "batched": pattern_batched, "adjoint": pattern_adjoint,
               "adjoint_fd": pattern_adjoint_fd,
               "relaxation": pattern_relaxation, "q1_2d": pattern_q1_2d, "renumber": pattern_renumber,
               "sharded": pattern_sharded, "steps": pattern_steps}[args.only]
        print(json.dumps({"pattern": args.only, **run(torch.cuda.current_stream(), args)}), flush=True)
        return
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    mesh = W.forward_step_mesh(m=args.m, jitter=0.2, seed=2007)
    U0 = W.forward_step_state(mesh)
    stream = torch.cuda.current_stream()
    s = Solver(mesh, stream=stream)
    s.init_state(U0)
    N, nnz = mesh.n_nodes, s.nnz

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up
    s.step(args.warmup)
    s.synchronize()

    # timed region: K SSP-RK3 steps with inputs resident in HBM
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except AttributeError:
        pass
    sampler = ClockSampler(bus_id=str(bus) if bus is not None else None)
    s.profile(True)
    barrier()
    torch.cuda.synchronize()
    if rank == 0:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    s.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if rank == 0 else None
    ms = e0.elapsed_time(e1)
    prof = s.profile_read()
    s.profile(False)
    ms_max, value = job_rate(ms, N * 3 * args.steps, dist, device="cuda")
    launches = sum(c for _, c in prof.values())

    # end-to-end through the public API with host buffers: every step copies
    # the state in from pinned host memory and the new state back out
    host_in = torch.from_numpy(U0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    s.init_state(host_in.numpy())
    s.step(1)
    s.get_state(host_out.numpy())
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.init_state(host_in.numpy())
        s.step(1)
        s.get_state(host_out.numpy())
        host_in, host_out = host_out, host_in
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    _, e2e_value = job_rate(e2e_s * 1e3, N * 3 * args.e2e_steps, dist, device="cuda")
    state_bytes = 5 * N * 8

    if rank == 0:
        peak64, peak64_src, peak64_clocks = fp64_peak(stream, str(bus) if bus is not None else None)
        dom = max(prof, key=lambda k: prof[k][0])
        dom_ms, dom_n = prof[dom]
        per_launch_s = dom_ms / dom_n * 1e-3
        achieved = FP64_FLOP_PER_NNZ_EXECUTED[dom] * nnz / per_launch_s / 1e12
        traffic = NCU_TRAFFIC_BYTES.get(dom) if args.m == 120 else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args.m, N, nnz, args),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak64,
                         "unit": "TFLOP/s", "frac": achieved / peak64, "traffic": traffic,
                         "peak_source": peak64_src, "peak_clocks": peak64_clocks,
                         "peak_derived_from_unit_counts": FP64_PEAK_TFLOPS,
                         "work": f"{FP64_FLOP_PER_NNZ_EXECUTED[dom]} executed FP64 flop/nnz (ncu, h = 1/80 after 3 warm-up steps) x {nnz} "
                                 f"nnz per launch",
                         "fp64_pipe_busy_ncu": FP64_PIPE_BUSY_NCU.get(dom),
                         "paper_flop_rate": FLOP_PER_NNZ[dom] * nnz / per_launch_s / 1e12},
            "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
            "kernels_share": {k: v[0] / sum(x[0] for x in prof.values()) for k, v in prof.items() if v[1]},
            "clocks": clocks,
        }
        exec_flops = sum(FP64_FLOP_PER_NNZ_EXECUTED.values())
        line["byte_model"] = byte_model(value, N, nnz, sum(NCU_TRAFFIC_BYTES.values()) if args.m == 120 else None,
                                        _hbm_peak()[0], peak64, exec_flops, "fp64")
        if not args.no_patterns:
            line["patterns"] = {"fp32_mixed": pattern_mixed(stream, args), "batched": pattern_batched(stream, args),
                                "adjoint": pattern_adjoint(stream, args),
                                "relaxation": pattern_relaxation(stream, args), "q1_2d": pattern_q1_2d(stream, args),
                                "renumber": pattern_renumber(stream, args), "sharded": pattern_sharded(stream, args)}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(mesh, U0, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
