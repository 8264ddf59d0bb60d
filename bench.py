"""Throughput of the FP64 WENO5-HLLC-SSP-RK3 step on one GB300 (or N independent replicas).

One "step" = one pass of the whole hot path over the grid: CFL reduction for dt, then three
Runge-Kutta stages, each = immersed-boundary ghost fill + domain halo fill + fused stage
kernel (WENO5, HLLC, viscous fluxes, divergence, stage combination).  The default workload is
the largest single-GPU configuration: the viscous Mach-2 shock over the immersed cylinder,
2048 x 1024 cells (Navier-Stokes, Re = 1000, Pr = 0.72).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload shock_cylinder|riemann2d|...]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
    python bench.py --workload mach5_cylinder --to-end   # one whole run to the end time
    python bench.py --to-end                             # the cylinder case's 2000 steps, per 250
    python bench.py --slabs 2,4 --steps 20               # the y-slab decomposition on one GPU

Prints ONE JSON line (rank 0).  `value` is cell-updates/s with the state resident in HBM;
`e2e` is the same metric through the C ABI with the state copied from pinned host memory
and back every step; `roofline` divides the algorithmic FP64 operation count of the stage
kernel by its CUDA-event time and by the FP64 peak.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Algorithmic FP64 operations (add/sub, mul, div, sqrt; each face once) per cell and RHS
# evaluation, counted by oracle/count_flops.py on a seeded perturbation of each workload.
FLOPS_PER_CELL_STAGE = {"riemann2d": 1281.0, "shock_cylinder": 1357.0, "mach5_cylinder": 1276.2}
# FP64 peak of one GB300: 152 SMs x 2070 MHz boost, NVIDIA's 1.25 TFLOP/s FP64 figure.
FP64_PEAK_TFLOPS = 1.25
# neural flux network per cell and stage: x and y face images, 2 x 6336 multiply-adds each
NN_FLOPS_PER_CELL_STAGE = 2 * 2 * 6336
# DRAM bytes (read + write) per stage-kernel launch, mean of the three stages of one step,
# from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of this bench's default
# run with the TMA-staged variant 0 and the current kernel; None for other workloads or
# variants (and for workloads whose capture predates the current kernel).
STAGE_TRAFFIC_BYTES = {("shock_cylinder", 0): 291.0e6, ("riemann2d", 0): 108.0e6}
# DRAM bytes per step of the persistent batched forward kernel on the 256-instance workload: an
# ncu capture of one 2-step launch of the current kernel (19.27 GB), scaled by the steps of a launch
BATCH_TRAFFIC_PER_STEP = 9.64e9
L2_FLUSH_BYTES = 256 << 20
METRIC = "FP64 cell-updates/s per RK step on 1 GB300 (% roofline); adjoint/forward time ratio"


def workload(name):
    from paper_2601_04400_gb300 import workloads as W
    if name == "riemann2d":
        p = W.riemann2d(1024)
        desc = "2D four-quadrant Riemann problem, Euler, 1024x1024, WENO5+HLLC+SSP-RK3, CFL 0.5, transmissive"
    elif name == "shock_cylinder":
        p = W.shock_cylinder()
        desc = ("viscous Mach-2 shock over an immersed cylinder, Navier-Stokes Re=1000 Pr=0.72, 2048x1024, "
                "WENO5+HLLC+IB+SSP-RK3, CFL 0.5")
    elif name == "mach5_cylinder":
        p = W.mach5_cylinder()
        desc = ("the paper's Mach-5 shock over an immersed cylinder, Euler, 4347x1932 (8.40e6 cells) on "
                "[-0.5,4]x[0,2], WENO5+HLLC+IB+SSP-RK3, CFL 0.5, inflow/outflow/reflective")
    else:
        raise SystemExit("unknown workload %s" % name)
    return p, desc


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to $JS_CLOCKS_CSV when set (to keep them), else to a temporary file
        self.path = os.environ.get("JS_CLOCKS_CSV")
        if not self.path:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)

    def __enter__(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(prob, budget_s=12.0):
    """The oracle, as it stands, on the host cores: full-grid SSP-RK3 steps for ~budget_s."""
    import oracle as O
    U = O.prim_to_cons(prob, prob.W0)
    dt = O.max_dt(prob, U, prob.cfl)
    steps, t0 = 0, time.perf_counter()
    while True:
        U = O.step(prob, U, [dt])
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 200:
            break
    return {"value": prob.cells * steps / el, "unit": "cell-updates/s", "cores": O.threads(), "kind": "oracle",
            "sample": "%d SSP-RK3 steps of the full %dx%d grid from the initial state, fixed dt, %.1f s"
                      % (steps, prob.nx, prob.ny, el)}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from oracle import build as ob
    ob.build()
    prob, desc = workload(args.workload)
    U = O.prim_to_cons(prob, prob.W0)
    dt = O.max_dt(prob, U, prob.cfl)
    t0 = time.perf_counter()
    U1 = O.step(prob, U, [dt])
    t1 = time.perf_counter() - t0
    # bound the whole run to about two and a half minutes: a band of rows around the
    # quadrant split when the full grid would take longer
    budget = 150.0
    rows = prob.ny
    if (args.steps + args.warmup) * t1 > budget:
        rows = max(16, int(prob.ny * budget / ((args.steps + args.warmup) * t1)))
    sub = prob
    if rows < prob.ny:
        j0 = max(0, min(prob.ny - rows, int(0.8 * prob.ny) - rows // 2))
        sub = prob.with_(ny=rows, y0=prob.y0 + j0 * prob.dy, W0=np.array(prob.W0[:, j0:j0 + rows]),
                         sdf=None if prob.sdf is None else np.array(prob.sdf[:, j0:j0 + rows]))
    Us = O.prim_to_cons(sub, sub.W0)
    for _ in range(args.warmup):
        Us = O.step(sub, Us, [dt])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Us = O.step(sub, Us, [dt])
    el = time.perf_counter() - t0
    value = sub.cells * args.steps / el
    sample = ("%d SSP-RK3 steps of a %dx%d %s of the workload, fixed dt" %
              (args.steps, sub.nx, sub.ny, "band" if rows < prob.ny else "grid"))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "nx": sub.nx, "ny": sub.ny},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": O.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    prob, desc = workload(args.workload)
    stream = torch.cuda.current_stream()
    solver = B.Solver.from_problem(prob, stream=stream)
    W0 = torch.tensor(prob.W0, dtype=torch.float64, device="cuda")
    U = solver.prim_to_cons(W0)
    from paper_2601_04400_gb300 import tuning
    tuned = tuning.autotune(solver, U)  # stage-kernel tile shape (identical results)
    U0 = U.clone()
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    cfl = prob.cfl

    def one_step(Ud):
        # CFL reduction, device step size and the three stages; no host synchronisation
        solver.step_cfl(Ud, cfl, 1)

    for _ in range(args.warmup):
        one_step(U)
    solver.check()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing -------------------------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    with sampler:
        B.js_profile_begin(solver.ctx, 3 * args.steps + 8)
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            one_step(U)
            ev[k][1].record(stream)
        stage_ms, stage_launches, launches = B.js_profile_end(solver.ctx)
        barrier()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    solver.check()
    # ---- end to end through the C ABI with host buffers -------------------------------
    Uh = torch.empty(U.shape, dtype=torch.float64).pin_memory()
    Uh.copy_(U0.cpu())
    Ud = torch.empty_like(U)
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ee[k][0].record(stream)
        Ud.copy_(Uh, non_blocking=True)
        one_step(Ud)
        Uh.copy_(Ud, non_blocking=True)
        ee[k][1].record(stream)
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in ee)
    solver.check()

    # ---- adjoint / forward cost of one SSP-RK3 step (same state, same dt) ---------------
    adj = None
    if not args.no_adjoint:
        dt = solver.max_dt(U, cfl)
        lam = torch.randn(U.shape, dtype=torch.float64, device="cuda")
        lam_out = torch.empty_like(lam)
        pbar = torch.zeros(20, dtype=torch.float64, device="cuda")
        Uw = U.clone()
        solver.step_vjp(U, dt, lam, lam_n=lam_out, p_bar=pbar)  # allocates the adjoint workspace
        reps = max(3, min(args.steps, 20))
        fa = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        ba = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        barrier()
        for k in range(reps):
            flush.zero_()
            fa[k][0].record(stream)
            solver.step(Uw, dt, 1)
            fa[k][1].record(stream)
            flush.zero_()
            ba[k][0].record(stream)
            solver.step_vjp(U, dt, lam, lam_n=lam_out, p_bar=pbar)
            ba[k][1].record(stream)
        barrier()
        solver.check()
        f_ms = sum(a.elapsed_time(b) for a, b in fa) / reps
        b_ms = sum(a.elapsed_time(b) for a, b in ba) / reps
        # reverse of a step whose stage states (and WENO internals) were recorded: the
        # checkpointed rollout's path; its backward re-runs each step taped, then reverses it
        solver.tape_reserve(1, weno=True)
        solver.step_taped(Uw, dt, 0)
        tf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        ta = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        barrier()
        for k in range(reps):
            Ut = U.clone()
            flush.zero_()
            tf[k][0].record(stream)
            solver.step_taped(Ut, dt, 0)
            tf[k][1].record(stream)
            flush.zero_()
            ta[k][0].record(stream)
            solver.step_vjp_taped(0, dt, lam, lam_n=lam_out, p_bar=pbar)
            ta[k][1].record(stream)
        barrier()
        solver.check()
        tf_ms = sum(a.elapsed_time(b) for a, b in tf) / reps
        t_ms = sum(a.elapsed_time(b) for a, b in ta) / reps
        adj = {"ms_per_step_forward": f_ms, "ms_per_step_vjp": b_ms, "ratio": b_ms / f_ms,
               "ms_per_step_taped_forward": tf_ms, "ms_per_step_vjp_taped": t_ms, "ratio_taped": t_ms / f_ms,
               "ratio_rollout_backward": (tf_ms + t_ms) / f_ms,
               "note": "ratio: js_step_vjp (recomputes the stage states, then reverses the 3 stages) / "
                       "js_step; ratio_taped: js_step_vjp_taped (stage states and WENO5 internals recorded "
                       "by js_step_taped) / js_step; ratio_rollout_backward: (js_step_taped + "
                       "js_step_vjp_taped) / js_step, the backward cost per step of a checkpointed rollout"}

    # ---- the workload's whole run (step-count workloads): every part of it, not only the start ----
    run = None
    if prob.n_steps and not args.no_whole_run:
        run = whole_run(prob, solver, U0.clone(), stream)
        run["note"] = ("the configuration's whole run from t = 0 (js_step_cfl in chunks of 250 steps, CUDA "
                       "events); `value` times the steps right after the initial condition")

    # ---- neural flux (Sec. 2.3): step and reverse step with the network, FP32 and FP64 -----
    neural = None
    if args.neural:
        from paper_2601_04400_gb300 import neural as NN
        w = NN.init_weights(0, zero_last=False) * 0.5
        norm = NN.frame_norm(U, scale=0.1)
        wb = torch.zeros_like(w)
        dt = solver.max_dt(U, cfl)
        lam = torch.randn(U.shape, dtype=torch.float64, device="cuda")
        lam_out = torch.empty_like(lam)
        pbar = torch.zeros(20, dtype=torch.float64, device="cuda")
        reps = max(3, min(args.steps, 10))
        neural = {"flops_per_cell_stage_network": NN_FLOPS_PER_CELL_STAGE,
                  "note": "network forward per stage: 2 face images (x faces, y faces) x 6336 multiply-adds "
                          "per face; ms per SSP-RK3 step with the network on, and the reverse step "
                          "(js_step_vjp with the weight gradient); bf16: the forward's three layers on the "
                          "tensor cores (BF16 operands, FP32 accumulation), the forward-only stages' network in one fused launch; "
                          "bf16-layerwise: the same arithmetic and results, one launch per layer"}
        for name in ("bf16", "bf16-layerwise", "fp32", "fp64"):
            solver.set_neural(w, norm, w_bar=wb, precision=name)
            Uw = U.clone()
            for _ in range(2):  # warm-up (the first calls allocate the network's workspaces)
                solver.step(Uw, dt, 1)
                solver.step_vjp(U, dt, lam, lam_n=lam_out, p_bar=pbar)
            fa = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            ba = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            barrier()
            for k in range(reps):
                flush.zero_()
                fa[k][0].record(stream)
                solver.step(Uw, dt, 1)
                fa[k][1].record(stream)
                flush.zero_()
                ba[k][0].record(stream)
                solver.step_vjp(U, dt, lam, lam_n=lam_out, p_bar=pbar)
                ba[k][1].record(stream)
            barrier()
            solver.check()
            f_ms = sum(a.elapsed_time(b) for a, b in fa) / reps
            b_ms = sum(a.elapsed_time(b) for a, b in ba) / reps
            neural[name] = {"ms_per_step": f_ms, "ms_per_step_vjp": b_ms,
                            "network_tflops_over_whole_step": 3 * NN_FLOPS_PER_CELL_STAGE * prob.cells / (f_ms * 1e-3) / 1e12}
        solver.set_neural(None)

    if dist is not None:
        t = torch.tensor([step_ms, e2e_ms, stage_ms / max(stage_launches, 1)], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms, e2e_ms, stage_avg = t.tolist()
    else:
        stage_avg = stage_ms / max(stage_launches, 1)
    cells = prob.cells
    value = world * cells * args.steps / (step_ms * 1e-3)
    e2e_value = world * cells * args.steps / (e2e_ms * 1e-3)
    flop_launch = FLOPS_PER_CELL_STAGE[args.workload] * cells
    achieved = flop_launch / (stage_avg * 1e-3) / 1e12
    state_bytes = 4 * cells * 8
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "nx": prob.nx, "ny": prob.ny, "cells": cells,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between steps (256 MiB write)",
                       "step": "CFL reduction + device step size + 3 x (IB fill, halo fill, fused stage "
                               "kernel) (js_step_cfl)",
                       "stage_variant": solver.tuning()[0]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": STAGE_TRAFFIC_BYTES.get((args.workload, solver.tuning()[0])),
                         "kernel": "stage2d (fused WENO5-HLLC stage)", "stage_ms_avg": stage_avg,
                         "flops_per_launch": flop_launch},
            "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes},
            "adjoint_forward_ratio": None if adj is None else adj["ratio"],
            "adjoint": adj,
            "whole_run": run,
            "neural": neural,
            "gpu_launches": launches,
            "clocks": sampler.summary(),
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(prob)
        print(json.dumps(out), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args):
    """Many independent shock-cylinder instances: one persistent launch per js_batch_step
    (device CFL per instance) against one-at-a-time js_max_dt + js_step per instance."""
    import torch
    from paper_2601_04400_gb300 import binding as B
    from paper_2601_04400_gb300 import workloads as W
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2601_04400_gb300 import parallel
    probs = W.batched_cases(args.instances, seed=0)
    # instances are sharded over ranks by cell count (no exchange between them)
    mine = [probs[k] for k in parallel.shard([p.cells for p in probs], world, rank)]
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    states = []
    for p in mine:
        s = B.Solver.from_problem(p, stream=stream)
        states.append(s.prim_to_cons(torch.tensor(p.W0, dtype=torch.float64, device="cuda")))
        s.close()
    cells = sum(p.cells for p in mine)
    batch = B.Batch(mine, stream=stream)
    from paper_2601_04400_gb300 import tuning
    tuned = tuning.autotune_batch(batch, mine, states)  # blocks per SM and schedule (identical results)
    work = [U.clone() for U in states]
    batch.set_states(work)
    batch.step(0.5, args.warmup)
    torch.cuda.synchronize()
    if batch.status() != 0:
        raise SystemExit("batched warm-up failed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    with sampler:
        e0.record(stream)
        batch.step(0.5, args.steps)  # one persistent launch for all steps
        e1.record(stream)
        e1.synchronize()
    t_batch = e0.elapsed_time(e1)
    ok = batch.status() == 0
    # end to end through the public API: every step copies all instance states in from pinned
    # host memory, advances them with js_batch_step and copies them back
    host = [U.detach().cpu().pin_memory() for U in work]
    torch.cuda.synchronize()
    e2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        e2[k][0].record(stream)
        for U, H in zip(work, host):
            U.copy_(H, non_blocking=True)
        batch.step(0.5, 1)
        for U, H in zip(work, host):
            H.copy_(U, non_blocking=True)
        e2[k][1].record(stream)
    torch.cuda.synchronize()
    t_e2e = sum(a.elapsed_time(b) for a, b in e2)
    ok = ok and batch.status() == 0
    state_bytes = sum(U.numel() * 8 for U in work)
    local_cells = cells
    if dist is not None:
        tt = torch.tensor([t_batch, t_e2e, float(cells)], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt[:2], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[2:], op=dist.ReduceOp.SUM)
        t_batch, t_e2e, cells = float(tt[0]), float(tt[1]), int(tt[2])
    # one at a time: each instance its own context and its own device CFL steps (js_step_cfl:
    # no host round trip), instance after instance; and the same launches captured into one
    # CUDA graph per step of all instances, replayed
    solvers = [B.Solver.from_problem(p, stream=stream) for p in mine]
    seq = [U.clone() for U in states]
    for s, U in zip(solvers, seq):
        s.step_cfl(U, 0.5, args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    for s, U in zip(solvers, seq):
        s.step_cfl(U, 0.5, args.steps)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1)
    gseq = [U.clone() for U in states]
    side = torch.cuda.Stream()  # a capture needs a stream of its own
    torch.cuda.synchronize()
    for s in solvers:
        s.set_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            for s, U in zip(solvers, gseq):
                s.step_cfl(U, 0.5, 1)
        torch.cuda.synchronize()
        e0.record(side)
        for _ in range(args.steps):
            graph.replay()
        e1.record(side)
        e1.synchronize()
    t_graph = e0.elapsed_time(e1)
    for s in solvers:
        s.set_stream(stream)
    ok = ok and all(s.status() == 0 for s in solvers)
    # reverse of one batched step (js_batch_step_vjp over all instances) against one batched
    # forward step, in both launch forms (one persistent launch; one launch per phase); the tuner
    # keeps the faster for the rollout below
    dts = [s.max_dt(U, 0.5) for s, U in zip(solvers, states)]
    lams = [torch.randn_like(U) for U in states]
    outs = [torch.empty_like(U) for U in states]
    rev_tuned = tuning.autotune_batch_reverse(batch, mine, states, dts)
    t_vjp_form = {}
    choice = batch.reverse_launch()
    reps = 3
    for split in (0, 1):
        batch.set_reverse_launch(split)
        batch.step_vjp(states, dts, lams, outs)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            batch.step_vjp(states, dts, lams, outs)
        e1.record(stream)
        e1.synchronize()
        t_vjp_form[split] = e0.elapsed_time(e1) / reps
    batch.set_reverse_launch(choice)
    t_vjp = t_vjp_form[choice]
    ok = ok and batch.status() == 0
    # the whole rollout: n_ro CFL steps forward (step sizes logged), then its reverse
    # (js_batch_rollout_vjp) with the library's checkpoint spacing (every state when they fit in
    # half the free device memory, else sqrt(N)); the first reverse call allocates its
    # workspace and is not timed
    n_ro = args.rollout_steps
    roll = None
    if n_ro > 0:
        log = torch.zeros((n_ro, len(mine)), dtype=torch.float64, device="cuda")
        lam_r = [torch.randn_like(U) for U in states]
        # first round: allocates the rollout workspace (not timed)
        batch.set_states([U.clone() for U in states])
        batch.rollout_forward(0.5, log)
        batch.rollout_vjp(log, lam_r)
        torch.cuda.synchronize()
        # the plain forward run of the same steps: one launch, device CFL
        batch.set_states([U.clone() for U in states])
        e0.record(stream)
        batch.step(0.5, n_ro, dt_log=log)
        e1.record(stream)
        e1.synchronize()
        t_ro_plain = e0.elapsed_time(e1)
        # the checkpointed forward and its reverse
        batch.set_states([U.clone() for U in states])
        e0.record(stream)
        batch.rollout_forward(0.5, log)
        e1.record(stream)
        e1.synchronize()
        t_ro_f = e0.elapsed_time(e1)
        e0.record(stream)
        batch.rollout_vjp(log, lam_r)
        e1.record(stream)
        e1.synchronize()
        t_ro_b = e0.elapsed_time(e1)
        ok = ok and batch.status() == 0
        ck = batch.rollout_spacing(n_ro)
        roll = {"steps": n_ro, "checkpoint_every": ck, "ms_forward_plain": t_ro_plain,
                "ms_forward_checkpointed": t_ro_f, "ms_reverse": t_ro_b, "ratio": t_ro_b / t_ro_plain,
                "note": "ratio: js_batch_rollout_vjp (per segment: re-run keeping its states and stage "
                        "states + the reverse of each step (the chosen launch form) taking the stage states as given, "
                        "from the checkpoints js_batch_rollout_forward kept; spacing 1 = every state and "
                        "stage state kept by the forward, no re-runs) / the plain batched forward run of "
                        "the same steps (one launch, device CFL)"}
    info = batch.info()
    if rank == 0:
        print(json.dumps({
            "metric": "FP64 cell-updates/s, batched shock-cylinder instances", "value": cells * args.steps / (t_batch * 1e-3),
            "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_batch / args.steps, "higher_is_better": True, "scaling": "weak", "dtype": "f64",
            "data": "synthetic", "status_ok": ok,
            "config": {"workload": "%d viscous shock-cylinder instances (seed 0: Mach U[1.5,3], radius U[0.3,0.7], "
                                   "nx 128..512, ny 128..256), per-instance device CFL 0.5" % len(mine),
                       "cells": cells, "persistent_blocks": info["blocks"], "tiles": info["tiles"],
                       "tuning": {"blocks_per_sm": batch.tuning()[0], "schedule": batch.tuning()[2],
                                  "timed": {"%d,%d" % k: v for k, v in tuned.items()}}},
            "e2e": {"value": cells * args.steps / (t_e2e * 1e-3), "unit": "cell-updates/s",
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
            "roofline": {"bound": "alu", "kernel": "batch_kernel (persistent: CFL, IB and halo fills, stage tiles)",
                         "achieved": FLOPS_PER_CELL_STAGE["shock_cylinder"] * 3 * cells * args.steps
                         / (t_batch * 1e-3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": FLOPS_PER_CELL_STAGE["shock_cylinder"] * 3 * cells * args.steps
                         / (t_batch * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "traffic": BATCH_TRAFFIC_PER_STEP * args.steps if args.instances == 256 and world == 1
                         else None,
                         "flops_per_cell_stage": FLOPS_PER_CELL_STAGE["shock_cylinder"]},
            "gpu_launches": 1, "clocks": sampler.summary(),
            "one_at_a_time": {"value": local_cells * args.steps / (t_seq * 1e-3), "ms_per_step": t_seq / args.steps,
                              "how": "rank 0's instances one after another, each js_step_cfl for all steps "
                                     "(device CFL, no host round trip)"},
            "one_at_a_time_graph": {"value": local_cells * args.steps / (t_graph * 1e-3),
                                    "ms_per_step": t_graph / args.steps,
                                    "how": "one CUDA graph holding one js_step_cfl step of every instance, "
                                           "replayed once per step"},
            "speedup_vs_one_at_a_time": t_seq / t_batch,
            "speedup_vs_graph": t_graph / t_batch,
            "adjoint": {"ms_per_step_vjp": t_vjp, "ratio": t_vjp / (t_batch / args.steps),
                        "launch": "one launch per phase" if choice else "one persistent launch",
                        "ms_per_step_vjp_persistent": t_vjp_form[0], "ms_per_step_vjp_split": t_vjp_form[1],
                        "tuner_timed": {str(k): v for k, v in rev_tuned.items()},
                        "note": "js_batch_step_vjp (recompute of the stage states and the reverse of the 3 "
                                "stages of every instance; the launch form the tuner chose) / one batched "
                                "forward step, rank 0's instances"},
            "rollout": roll}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_to_end(args):
    """A whole run of a single-grid workload from t = 0 to its end time with the CFL step (the
    last step before each output time clipped to it), timed with CUDA events around the loop: the
    wall time of the application, next to the paper's reported wall times (context only).  At the
    output times it reports the density range and the x position of the leading shock front on
    the bottom wall (the last cell of the bottom row whose density exceeds twice the undisturbed
    gas's)."""
    import torch
    from paper_2601_04400_gb300 import binding as B
    B.lib()
    prob, desc = workload(args.workload)
    stream = torch.cuda.current_stream()
    solver = B.Solver.from_problem(prob, stream=stream)
    U = solver.prim_to_cons(torch.tensor(prob.W0, dtype=torch.float64, device="cuda"))
    if prob.t_end is None:
        return run_steps_to_end(args, prob, desc, solver, U, stream)
    outputs = sorted(set([t for t in (0.3, 1.0) if t < prob.t_end] + [prob.t_end]))
    rho_far = float(np.min(prob.W0[0]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t, steps, snaps = 0.0, 0, []
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    e0.record(stream)
    for t_out in outputs:
        while t < t_out:
            dt = solver.max_dt(U, prob.cfl)
            last = t + dt >= t_out
            if last:
                dt = t_out - t
            solver.step(U, dt, 1)
            t = t_out if last else t + dt
            steps += 1
        r = U[0]
        bottom = (r[0] > 2.0 * rho_far).nonzero()
        front = float(prob.x0 + (int(bottom[-1]) + 0.5) * prob.dx) if bottom.numel() else None
        snaps.append({"t": t_out, "steps": steps, "rho_min": float(r.min()), "rho_max": float(r.max()),
                      "wall_shock_x": front})
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    status = solver.status()
    gpu_s = e0.elapsed_time(e1) * 1e-3
    cells = prob.nx * prob.ny
    print(json.dumps({"mode": "run_to_t_end", "workload": desc, "t_end": prob.t_end, "steps": steps,
                      "cells": cells, "seconds": gpu_s, "wall_seconds": wall,
                      "cell_updates_per_s": cells * steps / gpu_s, "dtype": "f64", "status_ok": status == 0,
                      "outputs": snaps}), flush=True)


def whole_run(prob, solver, U, stream, chunk=250):
    """The whole run of a workload defined by its step count (the viscous shock-cylinder case:
    2000 CFL steps from t = 0) with device-computed step sizes (js_step_cfl, no host round trip),
    in chunks timed with CUDA events: the throughput of every part of the run, from the quiescent
    start to the developed wake.  U is advanced in place."""
    import torch
    ev = []
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    done = 0
    while done < prob.n_steps:
        n = min(chunk, prob.n_steps - done)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solver.step_cfl(U, prob.cfl, n, t=t)
        b.record(stream)
        ev.append((done, n, a, b))
        done += n
    torch.cuda.synchronize()
    solver.check()
    cells = prob.nx * prob.ny
    gpu_s = sum(a.elapsed_time(b) for _, _, a, b in ev) * 1e-3
    return {"steps": prob.n_steps, "t_final": float(t), "seconds": gpu_s,
            "cell_updates_per_s": cells * prob.n_steps / gpu_s,
            "chunks": [{"first_step": d, "steps": n, "ms_per_step": a.elapsed_time(b) / n} for d, n, a, b in ev]}


def run_steps_to_end(args, prob, desc, solver, U, stream):
    """--to-end for a workload defined by its step count: one whole run, timed in chunks."""
    r = whole_run(prob, solver, U, stream)
    print(json.dumps({"mode": "run_n_steps", "workload": desc, "cells": prob.nx * prob.ny, "dtype": "f64", **r}),
          flush=True)


def run_slabs(args):
    """The single-grid workload decomposed into K y slabs held by this process (one GPU, the
    slabs' launches run one after another, so this times the decomposition's own cost: overlap
    rows, per-stage packing and exchange, not a multi-GPU step) next to the undecomposed step:
    forward step and reverse step (js_step_vjp against SlabGroup.step_vjp), ms per step."""
    import torch
    from paper_2601_04400_gb300 import binding as B
    from paper_2601_04400_gb300 import parallel
    B.lib()
    prob, desc = workload(args.workload)
    s = B.Solver.from_problem(prob)
    U0 = s.prim_to_cons(torch.tensor(prob.W0, dtype=torch.float64, device="cuda"))
    dt = 0.5 * s.max_dt(U0, prob.cfl)
    lam = torch.randn_like(U0)

    def timed(fn, n):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    U = U0.clone()
    out = {"mode": "slabs", "workload": desc, "dtype": "f64",
           "whole": {"ms_step": timed(lambda: s.step(U, dt, 1), args.steps),
                     "ms_step_vjp": timed(lambda: s.step_vjp(U0, dt, lam), max(1, args.steps // 4))}}
    periodic = prob.bc[2] == 2
    for k in sorted(set(int(v) for v in args.slabs.split(","))):
        plan = parallel.SlabPlan(prob.ny, k, args.overlap, periodic=periodic)
        G = parallel.SlabGroup.build(prob, plan, range(k))
        X, XU, XL = G.scatter(U0), G.scatter(U0), G.scatter(lam)
        out["slabs_%d" % k] = {"ms_step": timed(lambda: G.step(X, dt, 1), args.steps),
                               "ms_step_vjp": timed(lambda: G.step_vjp(XU, dt, XL), max(1, args.steps // 4)),
                               "overlap": plan.overlap}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shock_cylinder", choices=["riemann2d", "shock_cylinder", "mach5_cylinder", "batched"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--rollout-steps", type=int, default=60,
                    help="batched workload: steps of the rollout whose checkpointed reverse is timed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-whole-run", action="store_true",
                    help="skip the timing of the workload's whole run (step-count workloads)")
    ap.add_argument("--neural", action="store_true", help="also time steps with the neural flux")
    ap.add_argument("--to-end", action="store_true",
                    help="one whole run of the workload to its end time or step count (CFL steps), timed "
                         "as an application")
    ap.add_argument("--slabs", default=None,
                    help="comma-separated slab counts: time the y-slab decomposition held by this process")
    ap.add_argument("--overlap", type=int, default=3, help="overlap rows of the slabs (--slabs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.slabs and args.impl == "ours" and args.workload != "batched":
        run_slabs(args)
    elif args.to_end and args.impl == "ours" and args.workload != "batched":
        run_to_end(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
