#!/usr/bin/env python
"""Benchmark: explicit time steps per second of the semi-explicit eddy-current
time stepper (Schur-complement ODE, explicit Euler, one Jacobi-PCG solve of
K_n per step at relative residual 1e-10, SPE start vectors of depth 8) on the
64^3 Brauer-iron workload (24x24x16 iron block, sigma 2e6 S/m, 40x40 coil,
500 A at 50 Hz), FP64, one handle per GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` = time steps per second over the K timed steps
(device time of each step by CUDA events on the library's stream, L2 flushed
by a 256 MiB write between steps).  `e2e` = the same metric through the host
C ABI (state in and out of pinned host memory every step, wall clock).
With N > 1 (torchrun) every rank advances an independent replica (no data
exchange: the single-instance path does not shard) and `value` counts the
steps of all ranks over the slowest rank's time.  `--impl reference` times the
FP64 CPU oracle (the correctness reference) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "explicit time steps/sec and PCG iters/step at rel-residual 1e-10; stencil HBM GB/s vs peak"
WORKLOAD = "nonlinear-iron-64^3 (Brauer iron 24x24x16, sigma 2e6 S/m, coil 40x40 at z=32, 500 A 50 Hz)"


def workload_name(p):
    """Name of a scaled iron workload, from its description."""
    import numpy as np
    if p.N == 64:
        return WORKLOAD
    nz = np.nonzero(p.sigma_cell)
    ext = [int(a.max() - a.min() + 1) for a in (nz[2], nz[1], nz[0])]
    sig = float(p.sigma_cell[nz].max())
    return (f"nonlinear-iron-{p.N}^3 (Brauer iron {ext[0]}x{ext[1]}x{ext[2]}, sigma {sig:.0e} S/m, "
            f"coil {p.coil_i1 - p.coil_i0}x{p.coil_j1 - p.coil_j0} at z={p.coil_k}, {p.amplitude:g} A 50 Hz)")
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz
FLOPS_PER_ITER = 16                                   # stencil 6 adds + 5 FMAs, per unknown
FLOPS_PER_RESIDUAL = 9                                # stencil 6 + subtract 1 + FMA 2, per unknown
# algorithmic bytes per unknown and PCG iteration: x, r, p read and written once, at the
# value size of the iteration's vectors (FP64 and float-float: 8 B; FP32 inner CG: 4 B)
BYTES_PER_ITER = {0: 48, 1: 24, 2: 48}
PRECISION_NAMES = {
    0: "FP64 (PCG, stencil, conductor update, residuals); SPE difference table, its Galerkin products and "
       "x0 = D y in float-float (FP32 pairs, about 48 bits)",
    1: "FP32 inner CG in FP64 refinement (FP64 residual, update and stopping test); SPE table in float-float",
    2: "float-float inner CG in FP64 refinement (FP64 residual, update and stopping test); SPE table in "
       "float-float"}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 FMA lanes/clk x 2 flop x 2070 MHz
# DRAM bytes of the PCG kernel on the 64^3 iron workload from one ncu capture of the current
# kernel build (a zero-start solve of 221 iterations, profiles/pcg_fused_kernel_...): bytes
# read per launch (the carried vectors stay in L2) and bytes written per iteration (L2
# write-back of the ping-pong vectors, which grows with the iterations); keyed by
# (precision, pcg_variant, halo warps per tile group).  A launch of the benchmark is scaled by
# its iteration count.
PCG_TRAFFIC = {(0, 1, 2): (12.924672e6, 241.222400e6 / 221)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------------------
def oracle_sample(warmup: int, steps: int, budget_s: float, dt: float):
    """Time the FP64 oracle on the workload: `warmup` untimed explicit Euler steps from
    rest, then up to `steps` timed ones (SPE depth 8, tol 1e-10, step dt), stopping early
    once `budget_s` seconds of timed steps are used: the steps the GPU arm times."""
    import numpy as np
    import oracle as O
    import workloads as W
    p = W.config_nonlinear_iron()
    t0 = time.perf_counter()
    d = O.Discretization(p)
    setup = time.perf_counter() - t0
    hist, a_c, its, done = [], None, [], 0
    for m in range(warmup):
        r = O.run_explicit_euler(d, dt, 1, start_mode=O.stepper.START_SPE, spe_depth=8, tol=1e-10,
                                 a_c0=a_c, m0=m, history=hist)
        a_c = r.a_c
    t1 = time.perf_counter()
    for m in range(warmup, warmup + steps):
        r = O.run_explicit_euler(d, dt, 1, start_mode=O.stepper.START_SPE, spe_depth=8, tol=1e-10,
                                 a_c0=a_c, m0=m, history=hist)
        a_c = r.a_c
        its.append(int(r.iterations[0]))
        done += 1
        if time.perf_counter() - t1 > budget_s:
            break
    el = time.perf_counter() - t1
    return {"steps_per_s": done / el, "steps": done, "first_step": warmup + 1, "seconds": el, "setup_s": setup,
            "iters_per_step": float(np.mean(its)), "threads": 1, "dt": dt}


def oracle_cmd(warmup, steps, budget_s, dt):
    return [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(steps), "--oracle-warmup",
            str(warmup), "--oracle-budget", str(budget_s), "--oracle-dt", repr(dt)]


ORACLE_ENV = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def run_oracle_subprocess(warmup, steps, budget_s, dt):
    """One single-thread oracle sample in a fresh interpreter (nothing forked from a
    process that holds a CUDA context)."""
    res = subprocess.run(oracle_cmd(warmup, steps, budget_s, dt), capture_output=True, text=True, env=ORACLE_ENV,
                         cwd=ROOT)
    if res.returncode != 0:
        raise RuntimeError("oracle sample failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_all_cores(warmup, steps, budget_s, dt):
    """The same single-thread oracle sample in one fresh interpreter per host core, all at
    once: the host's aggregate oracle throughput (independent trajectories; the oracle's
    sparse products do not scale over threads within one trajectory)."""
    cores = host_cores()
    procs = [subprocess.Popen(oracle_cmd(warmup, steps, budget_s, dt), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=ORACLE_ENV, cwd=ROOT) for _ in range(cores)]
    outs = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return {"value": sum(o["steps_per_s"] for o in outs), "cores": cores, "processes": cores,
            "per_process_steps_per_s": [o["steps_per_s"] for o in outs], "steps_each": outs[0]["steps"]}


def reference_dt():
    """The workload's step 0.9 * 2 / lambda_max with lambda_max from the oracle's power
    method (stored by tests/golden/make_golden.py --iron64)."""
    with open(os.path.join(ROOT, "tests", "golden", "nonlinear_iron_64.json")) as f:
        g = json.load(f)
    return g["dt"], g["lambda_max"]


# ----------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.lines = []
        self.proc = None
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if gpu_id:
                cmd += ["-i", gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def reduce_max(value, dist, device=None):
    """Maximum of a float over ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ----------------------------------------------------------------------------------------
def run_reference(args, rank, ws, dist):
    """The FP64 oracle on the host cores, on the GPU arm's workload, step and step range:
    warm-up steps untimed, then the timed steps (bounded by --reference-budget seconds),
    one thread; the line's `value` is that single-trajectory rate."""
    if rank != 0:
        return
    dt, lam = reference_dt()
    budget = float(args.reference_budget)
    s = run_oracle_subprocess(args.warmup, args.steps, budget, dt)
    sample = (f"explicit Euler steps {s['first_step']}..{s['first_step'] + s['steps'] - 1} of the workload from "
              f"rest (the steps the GPU arm times; {args.warmup} untimed warm-up steps before them), "
              f"dt {dt:.6e} s, SPE 8, tol 1e-10, one host thread, setup {s['setup_s']:.1f} s excluded"
              + ("" if s["steps"] == args.steps else f"; stopped after {s['steps']} of {args.steps} steps "
                 f"at the {budget:.0f} s budget"))
    line = {"impl": "reference", "metric": METRIC, "value": s["steps_per_s"], "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / s["steps_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": 64, "start_vector": "spe8", "tol": 1e-10, "dt_s": dt,
                       "lambda_max": lam, "dt_from": "0.9 * 2 / lambda_max, oracle power method",
                       "steps_timed": s["steps"], "first_step": s["first_step"]},
            "iters_per_step": s["iters_per_step"],
            "cpu_baseline": {"value": s["steps_per_s"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": s["steps_per_s"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(s, steps, warmup, stream, flush, dev):
    """Per-step device spans of `steps` queued steps (L2 flushed before each, CUDA events
    in stream order around each), after `warmup` untimed steps: (ms total, stats)."""
    import torch
    with torch.cuda.stream(stream):
        if warmup:
            s.step(warmup)
        torch.cuda.synchronize(dev)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            s.step_enqueue(1)
            ends[k].record(stream)
        _, sts = s.step_finish(steps, allow_fail=True)
        torch.cuda.synchronize(dev)
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)), sts


def graph_replay(args, s, stream, flush, dev, iters):
    """The timed steps once more from the same start (rest, the same warm-up), each
    steady-state step replayed from a CUDA graph and no event marks inside the steps:
    the arithmetic is bitwise the same, so the iterations repeat exactly and the
    difference in time is the cost of issuing the launches."""
    import numpy as np
    import torch
    s.set_state(np.zeros(s.n_c), 0.0, 0)
    s.reset_history()
    with torch.cuda.stream(stream):
        if args.warmup:
            s.step(args.warmup)
    g0 = s.graph_steps()
    ms, sts = timed_steps(s, args.steps, 0, stream, flush, dev)
    return {"ms": ms, "ms_per_step": ms / args.steps, "unit": "steps/s", "graph_steps": s.graph_steps() - g0,
            "same_iterations": [x.iterations for x in sts] == list(iters),
            "note": "the timed steps again from rest after the same warm-up, steady-state SPE steps "
                    "replayed from CUDA graphs (bitwise the same results)"}


def other_arithmetic(args, p, dt, stream, flush, dev):
    """The same workload and timing on the FP64-refined paths with FP32 and float-float
    inner solves (same tolerance on the FP64 true residual), each from rest."""
    import paper_1611_06721_gb300 as pkg
    out = {}
    for name, prec, var in (("f32+f64", 1, 1), ("ff+f64", 2, 1)):
        so = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, start_mode=pkg.START_SPE, spe_depth=8,
                                                          dt=dt, precision=prec, pcg_variant=var,
                                                          halo_warps=args.halo_warps, graph=args.graph))
        so.set_stream(stream.cuda_stream)
        ms, sts = timed_steps(so, args.steps, args.warmup, stream, flush, dev)
        so.close()
        out[name] = {"value": args.steps / (ms * 1e-3), "unit": "steps/s", "ms_per_step": ms / args.steps,
                     "iters_per_step": sum(x.iterations for x in sts) / len(sts),
                     "failed_steps": sum(1 for x in sts if x.status != 0),
                     "halo_warps": max(args.halo_warps, 1) if (prec, var) == (1, 1) and p.N < 96 else 1}
    return out


def run_ours(args, rank, ws, local, dist):
    # the batched measurement spreads its problems over 32 streams; CUDA maps streams onto
    # this many hardware queues (read when the context is created)
    if args.batch_sub > 0:
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = W.config_nonlinear_iron() if args.grid == 64 else W.scaled_nonlinear(args.grid)
    mode = {"zero": pkg.START_ZERO, "prev": pkg.START_PREV, "spe": pkg.START_SPE, "pod": pkg.START_POD,
            "cspe": pkg.START_CSPE}[args.start]
    depth = args.depth if args.depth else {"spe": 8, "cspe": 16}.get(args.start, 20)
    opts = pkg.SolverOptions(tol=1e-10, start_mode=mode,
                             spe_depth=depth if args.start in ("spe", "cspe") else 8,
                             pod_snapshots=depth if args.start == "pod" else 20, pcg_variant=args.pcg_variant,
                             halo_warps=args.halo_warps, cspe_period=args.cspe_period,
                             precision=args.precision, rhs_split=1 if args.rhs_split else 0,
                             eps_lin=args.eps_lin, graph=args.graph)
    s = pkg.Solver.from_problem(p, opts)
    stream = torch.cuda.Stream(device=dev)
    s.set_stream(stream.cuda_stream)
    # setup: dt = 0.9 * 2 / lambda_max(M_c^-1 K_S) by the power method (eq. (CFL))
    t0 = time.perf_counter()
    if args.dt > 0:
        lam, pit, dt = None, 0, args.dt                    # given step (no power method)
    else:
        lam, pit = s.lambda_max(W.power_start_vector(s.n_c), pcg_tol=1e-12, rtol=1e-8, maxit=args.power_maxit)
        dt = 0.9 * 2.0 / lam
    s.set_dt(dt)
    setup_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        if args.warmup:
            s.step(args.warmup)
        torch.cuda.synchronize(dev)
        barrier(dist, dev)
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = None
        clocks = ClockSampler(gpu_id)
        s.timing_enable(True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        iters, statuses, refs = [], [], []
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            s.step_enqueue(1)
            ends[k].record(stream)            # in stream order: the step's device span
        # one finish for all steps: the host queues ahead and never idles the device
        rc, sts = s.step_finish(args.steps, allow_fail=True)
        for st in sts:
            iters.append(st.iterations)
            statuses.append(st.status)
            refs.append(st.refinements)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        tm = s.timing_get()
        s.timing_enable(False)
        barrier(dist, dev)
        graph = graph_replay(args, s, stream, flush, dev, iters) if args.graph and args.start == "spe" \
            and not args.rhs_split else None
        if graph:
            graph["value"] = ws * args.steps / (reduce_max(graph.pop("ms"), dist, dev) * 1e-3)
    ms_max = reduce_max(ms, dist, dev)
    value = ws * args.steps / (ms_max * 1e-3)
    # end to end through the host C ABI over the same steps: from rest, the same warm-up,
    # then each timed step with its state in from pinned host memory and out again, L2
    # flushed before each (outside its host-timed span)
    e2e = None
    if args.e2e:
        a_host = torch.empty(s.n_c, dtype=torch.float64, pin_memory=True).numpy()
        s.set_state(np.zeros(s.n_c), 0.0, 0)
        s.reset_history()
        with torch.cuda.stream(stream):
            if args.warmup:
                s.step(args.warmup)
            a_cur, t_cur, m_cur = s.get_state()
            a_host[:] = a_cur
            torch.cuda.synchronize(dev)
            barrier(dist, dev)
            el, e2e_its = 0.0, []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                t1 = time.perf_counter()
                s.set_state(a_host, t_cur, m_cur)
                _, st1 = s.step(1, allow_fail=True)
                _, t_cur, m_cur = s.get_state(out=a_host)
                el += time.perf_counter() - t1
                e2e_its.append(st1[0].iterations)
        el_max = reduce_max(el, dist, dev)
        e2e = {"value": ws * args.steps / el_max, "unit": "steps/s", "h2d_bytes_per_step": 8 * s.n_c,
               "d2h_bytes_per_step": 8 * s.n_c + 48, "steps": args.steps,
               "iters_per_step": float(np.mean(e2e_its)),
               "same_iterations": e2e_its == list(iters),
               "note": "the timed steps again from rest after the same warm-up, each through the host C ABI "
                       "(mqs_set_state from pinned memory, mqs_step, mqs_get_state), host wall clock per step, "
                       "L2 flushed before each step outside its span"}
    n_n = s.n_n
    its = np.array(iters)
    flops = n_n * (FLOPS_PER_ITER * its.sum() + 2 * FLOPS_PER_RESIDUAL * len(its))
    if args.precision != 0:
        # inner iterations plus one FP64 residual per refinement
        flops = n_n * (FLOPS_PER_ITER * its.sum() + FLOPS_PER_RESIDUAL * (len(its) + sum(refs)))
    achieved = flops / (tm["ms_pcg"] * 1e-3) / 1e12
    traffic = args.traffic
    # the capture is of the 64^3 workload: other grids get no traffic figure
    if traffic is None and args.grid == 64 and args.start == "spe" and depth == 8 and \
            (args.precision, args.pcg_variant, max(args.halo_warps, 1)) in PCG_TRAFFIC:
        rd, wr_it = PCG_TRAFFIC[(args.precision, args.pcg_variant, max(args.halo_warps, 1))]
        traffic = rd + wr_it * float(its.mean())
    if args.precision == 0:
        roof = {"bound": "alu", "kernel": "pcg_kernel" if args.pcg_variant == 0
                else f"pcg_fused_kernel<2,{max(args.halo_warps, 1)}>",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "note": "FP64 FMA=2 flop; peak derived: 152 SM x 2 FMA/clk x 2 x 2070 MHz"}
    else:
        roof = {"bound": "alu", "kernel": "pcg_mixed_kernel" if args.precision == 1 else "pcg_ff_kernel",
                "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": traffic,
                "note": "inner iterations (FP32 or float-float) against the FP32 issue peak (152 SM x 128 FMA/clk"
                        " x 2 x 2070 MHz); the inner iteration is latency and grid-barrier bound"}
    hbm = n_n * BYTES_PER_ITER[args.precision] * its.sum() / (tm["ms_pcg"] * 1e-3) / 1e9
    peaks = measured_peaks()
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f64", 1: "f32+f64", 2: "ff+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": workload_name(p), "grid": p.N, "n_unknowns": int(n_n), "n_conducting": int(s.n_c),
                       "precision": PRECISION_NAMES[args.precision],
                       "start_vector": args.start + (str(depth) if args.start in ("spe", "pod", "cspe") else "")
                                       + (f"/period {args.cspe_period or 25}" if args.start == "cspe" else ""),
                       "tol": 1e-10, "eps_lin": args.eps_lin, "dt_s": dt, "lambda_max": lam,
                       "pcg": ("one reduction per iteration" if (args.pcg_variant == 1 or args.precision == 2)
                               else "two reductions per iteration")
                              + (f", {max(args.halo_warps, 1)} halo warp(s) per tile group"
                                 if args.pcg_variant == 1 and args.precision == 0 else ""),
                       "right_hand_sides": "separate (conductor and coil types, one history each)" if args.rhs_split
                                           else "fused (one solve per step)",
                       "l2": "flushed between timed steps by a 256 MiB write",
                       "step_issue": "launch by launch, event marks between the phases",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "iters_per_step": float(its.mean()),
            "phases_ms_per_step": {k: tm[k] / args.steps for k in ("ms_rhs", "ms_start", "ms_pcg",
                                                                     "ms_conductor", "ms_history")},
            "roofline": roof,
            "stencil_hbm_view": {"algorithmic_GBps": hbm, "peak_GBps": peaks.get("hbm_gbs"),
                                 "frac": hbm / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                                 "note": f"{BYTES_PER_ITER[args.precision]} B/unknown/iteration (x, r, p read "
                                         "and written once)" + ("; the 64^3 PCG working set is L2-resident"
                                                                if p.N <= 64 else "")},
            "clocks": clk, "gpu_launches": int(tm["launches"]), "pcg_launches": int(tm["pcg_launches"]),
            "failed_steps": int(sum(1 for x in statuses if x != 0)),
            "setup": {"power_iterations": pit, "seconds": setup_s}}
    if e2e:
        line["e2e"] = e2e
    if graph:
        line["graph_replay"] = graph
    if ws == 1 and args.alt and args.start == "spe" and depth == 8 and args.precision == 0 and not args.rhs_split:
        line["other_arithmetic"] = {
            "note": "same workload and timing, FP64-refined PCG with FP32 / float-float inner solves to the same "
                    "1e-10 FP64 true residual (the headline value stays the FP64 path)",
            **other_arithmetic(args, p, dt, stream, flush, dev)}
    if rank == 0 and ws == 1 and not args.no_cpu and args.grid == 64:
        try:
            c = run_oracle_subprocess(args.warmup, args.steps, args.cpu_budget, dt)
            line["cpu_baseline"] = {
                "value": c["steps_per_s"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                "dt_s": dt, "iters_per_step": c["iters_per_step"],
                "sample": f"explicit Euler steps {c['first_step']}..{c['first_step'] + c['steps'] - 1} of the same "
                          f"workload (the steps timed above, {args.warmup} untimed warm-up steps before them), "
                          f"this line's dt, SPE 8, tol 1e-10, one host thread, setup excluded"}
            if args.cpu_all_cores:
                allc = run_oracle_all_cores(args.warmup, min(args.steps, 4), args.cpu_budget, dt)
                line["cpu_baseline"]["all_cores"] = {
                    "value": allc["value"], "unit": "steps/s", "cores": allc["cores"],
                    "sample": f"one single-thread oracle process per host core ({allc['processes']}), each "
                              f"stepping the same workload from rest and timing steps {args.warmup + 1}.."
                              f"{args.warmup + allc['steps_each']}: the host's aggregate throughput over "
                              f"independent trajectories"}
        except Exception as e:  # the GPU line is still valid without it
            line["cpu_baseline"] = {"value": None, "unit": "steps/s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e}"[:200]}
    s.close()
    if ws == 1 and args.batch_sub > 0:
        try:
            line["batch"] = batch_sub(args, dev)
        except Exception as e:  # the headline stays valid without it
            line["batch"] = {"failed": f"{e}"[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def coil_rhs(p, amp=100.0):
    """Right-hand side amp * X_s (the coil loop) in the device layout."""
    import numpy as np
    n = p.N
    b = np.zeros(3 * n ** 3)
    k = p.coil_k
    for i in range(p.coil_i0, p.coil_i1):
        b[i + n * (p.coil_j0 + n * k)] += amp
        b[i + n * (p.coil_j1 + n * k)] -= amp
    for j in range(p.coil_j0, p.coil_j1):
        b[n ** 3 + p.coil_i1 + n * (j + n * k)] += amp
        b[n ** 3 + p.coil_i0 + n * (j + n * k)] -= amp
    return b


def single_solve(variant=1, halo_warps=0):
    """One zero-start PCG solve of K_n w = 100 X_s on the workload (twice)."""
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    p = W.config_nonlinear_iron()
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(start_mode=pkg.START_ZERO, dt=1e-7, pcg_variant=variant,
                                                     halo_warps=halo_warps))
    b = coil_rhs(p)
    for _ in range(2):
        x, info = s.pcg_solve(b, tol=1e-10)
    print(json.dumps({"iterations": info.iterations, "relres": info.relres}))
    s.close()


def block_sweep(sizes):
    """What the batched mode can gain, per grid size: one zero-start solve of K_n w = 100 X_s
    on the scaled iron workload with the persistent PCG kernel on b blocks (b from 2 to one
    per SM), FP64 and FP32-inner (pcg_variant 1), CUDA-event time per iteration and its
    block-microseconds (b x time per iteration: constant where each block's share of the
    sweep sets the pace, rising where the grid reductions and barriers do).  A batch that
    runs its problems side by side on b_i blocks each can gain at most the ratio of the
    block-microseconds at one block per SM to those at b_i.  One JSON line per (size,
    precision)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    for n in sizes:
        p = W.config_nonlinear_iron() if n == 64 else W.scaled_nonlinear(n)
        for prec in (0, 1):
            s = pkg.Solver.from_problem(p, pkg.SolverOptions(start_mode=pkg.START_ZERO, dt=1e-7, precision=prec,
                                                             pcg_variant=1))
            stream = torch.cuda.Stream(device=dev)
            s.set_stream(stream.cuda_stream)
            b = torch.from_numpy(coil_rhs(p)).to(dev)
            x = torch.zeros_like(b)
            rows = []
            for nblk in (2, 4, 8, 16, 19, 38, 76, nsm):
                s.set_blocks(nblk)
                times = []
                for rep in range(2):                                 # the first is a warm-up
                    x.zero_()
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    info = s.pcg_solve_dev(b, x, tol=1e-10, stream=stream.cuda_stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
                its = max(info.iterations, 1)
                rows.append({"blocks": nblk, "iterations": info.iterations, "us_per_iter": 1e3 * times[-1] / its,
                             "block_us_per_iter": nblk * 1e3 * times[-1] / its})
            print(json.dumps({"sweep": "blocks per solve", "workload": workload_name(p), "grid": n,
                              "precision": "FP64" if prec == 0 else "FP32 inner CG in FP64 refinement",
                              "n_unknowns": int(s.n_n), "rows": rows}), flush=True)
            s.close()


def size_sweep(sizes):
    """Zero-start solves of K_n w = 100 X_s on the scaled iron workload at each grid
    size, FP64 and mixed precision (one-reduction FP32 inner CG): time per PCG
    iteration and the algorithmic bytes an iteration moves (x, r, p read and written
    once: 48 B per unknown in FP64, 24 B in FP32), against the measured copy bandwidth.
    The 64^3 vectors stay in L2; from 128^3 on the carried vectors exceed it.  One
    JSON line per (size, precision)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = measured_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for n in sizes:
        p = W.config_nonlinear_iron() if n == 64 else W.scaled_nonlinear(n)
        for prec, var, groups, halo in ((0, 1, 0, 0), (0, 1, 3, 0), (0, 1, 0, 2), (1, 1, 0, 0), (1, 1, 0, 2),
                                        (1, 2, 0, 0)):
            s = pkg.Solver.from_problem(p, pkg.SolverOptions(start_mode=pkg.START_ZERO, dt=1e-7, precision=prec,
                                                             pcg_variant=var, tile_groups=groups, halo_warps=halo))
            stream = torch.cuda.Stream(device=dev)
            s.set_stream(stream.cuda_stream)
            with torch.cuda.stream(stream):
                b = torch.from_numpy(coil_rhs(p)).to(dev)
                x = torch.zeros_like(b)
                s.pcg_solve_dev(b, x, tol=1e-10, stream=stream.cuda_stream)      # warm-up
                times, its = [], 0
                for _ in range(3):
                    x.zero_()
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    info = s.pcg_solve_dev(b, x, tol=1e-10, stream=stream.cuda_stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
                    its = info.iterations
            ms = statistics.median(times)
            us_it = 1e3 * ms / max(its, 1)
            gbs = BYTES_PER_ITER[prec] * s.n_n / (us_it * 1e-6) / 1e9
            print(json.dumps({"sweep": "zero-start solve", "workload": workload_name(p), "grid": n,
                              "precision": "FP64" if prec == 0 else "FP32 inner CG in FP64 refinement",
                              "pcg_variant": var, "tile_groups": groups or 2, "halo_warps": halo or 1,
                              "n_unknowns": int(s.n_n), "iterations": int(its), "relres": info.relres,
                              "status": int(info.status), "ms_per_solve": ms, "us_per_iteration": us_it,
                              "algorithmic_GBps": gbs, "hbm_peak_GBps": peaks.get("hbm_gbs"),
                              "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None}), flush=True)
            s.close()
            del b, x
            torch.cuda.empty_cache()


def run_batch(args):
    """Batched multi-query: `args.batch` independent instances (N from {32, 40, 48, 64},
    sigma ~ U[1e6, 5e6] S/m, amplitude ~ U[100, 1000] A, Brauer iron; seeded) advanced
    together (one stream each, PCG block counts proportional to the unknowns, the scale
    picked by the batch's tuner during warm-up).  value = instance-steps per second
    over the timed steps (device time from the fork of the streams to their join);
    the baseline is every instance stepped alone with all SMs (device time per step,
    a sample of steps each), as a plain loop over instances would run them."""
    # the batch spreads its problems over 32 streams; CUDA maps streams onto this many
    # hardware queues (read when the context is created)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sizes = tuple(int(v) for v in args.batch_grid.split(",")) if args.batch_grid else (32, 40, 48, 64)
    probs = W.batched_instances(args.batch, sizes=sizes)
    t0 = time.perf_counter()
    # lambda_max of M_c^-1 K_S per grid size at sigma 2e6 (power method, eq. (CFL)); M_c is
    # linear in sigma and K_S does not depend on it, so lambda_max scales as 1/sigma
    lam_ref = {}
    for n in sorted({p.N for p in probs}):
        s = pkg.Solver.from_problem(W.scaled_nonlinear(n), pkg.SolverOptions(tol=1e-10))
        lam_ref[n], _ = s.lambda_max(W.power_start_vector(s.n_c), pcg_tol=1e-12, rtol=1e-8,
                                     maxit=args.power_maxit)
        s.close()
    solvers = []
    for p in probs:
        sig = float(p.sigma_cell.max())
        lam = lam_ref[p.N] * 2.0e6 / sig
        solvers.append(pkg.Solver.from_problem(p, pkg.SolverOptions(
            tol=1e-10, start_mode=pkg.START_SPE, spe_depth=8, precision=args.precision,
            pcg_variant=args.pcg_variant, dt=0.9 * 2.0 / lam, graph=args.graph)))
    setup_s = time.perf_counter() - t0
    batch = pkg.Batch(solvers)
    best = batch.tune(max(args.warmup // 8, 1))      # 8 trials (4 scales, twice)
    by_work = batch.weighting()
    forms = batch.tune_pcg(args.tune_pcg_trials) if args.tune_pcg else [s_.pcg_form() for s_ in solvers]   # PCG kernel form per grid size
    form_by_n = {int(p.N): {"pcg_variant": int(v[0]), "tile_groups": int(v[1]), "halo_warps": int(v[2])}
                 for p, v in zip(probs, forms)}
    depth_by_n = None
    if args.tune_depth:
        chosen = batch.tune_depth(max(args.warmup // 4, 5), depths=(4, 8, 16))
        depth_by_n = {int(p.N): int(d) for p, d in zip(probs, chosen)}
    batch.step(args.warmup)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    g0 = batch.graph_steps()
    rc, stats = batch.step(args.steps, allow_fail=True)
    clk = clocks.stop()
    ms = batch.last_ms()
    graph_steps = batch.graph_steps() - g0
    batch.close()
    its = np.array([[x.iterations for x in row] for row in stats], dtype=float)
    failed = int(sum(1 for row in stats for x in row if x.status != 0))
    value = len(solvers) * args.steps / (ms * 1e-3)
    # baseline: each instance alone on the whole GPU
    stream = torch.cuda.Stream(device=dev)
    per_step_ms = []
    sample = max(min(args.steps // 5, 50), 5)
    for s in solvers:
        s.set_stream(stream.cuda_stream)
        s.step(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(sample)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        per_step_ms.append(e0.elapsed_time(e1) / sample)
        s.set_stream(0)
    seq = len(solvers) / (sum(per_step_ms) * 1e-3)
    sizes = {n: sum(1 for p in probs if p.N == n) for n in sorted({p.N for p in probs})}
    line = {"metric": "batched explicit time steps/sec (instance-steps) at rel-residual 1e-10",
            "value": value, "unit": "instance-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {0: "f64", 1: "f32+f64", 2: "ff+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{len(solvers)} instances, N from {set(sizes)} "
                                   f"(count per N {sizes}), sigma U[1e6,5e6] S/m, coil 100-1000 A, "
                                   f"Brauer iron, "
                                   + (f"SPE depth tuned per N {depth_by_n}" if depth_by_n else "SPE 8")
                                   + ", seed 1611",
                       "n_unknowns": int(sum(s.n_n for s in solvers)),
                       "precision": "FP64" if args.precision == 0 else "FP32 inner CG in FP64 refinement",
                       "blocks_scale": best, "block_shares": "unknowns x iterations" if by_work else "unknowns",
                       "pcg_form_by_N": form_by_n,
                       "l2": "working set larger than L2 (no flush)",
                       "graph_steps": graph_steps,
                       "parallelism": "1 GPU, instances on 32 streams"},
            "iters_per_step": float(its.mean()), "failed_steps": failed,
            "single_instance": {"value": seq, "unit": "instance-steps/s",
                                "note": f"each instance alone with all SMs, {sample} steps each"},
            "speedup_vs_single_instance": value / seq,
            "clocks": clk, "setup": {"seconds": setup_s, "lambda_ref": lam_ref}}
    print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()


def batch_sub(args, dev):
    """Batched multi-query beside the headline (the workload of the batched configuration,
    shortened): `args.batch_sub` seeded instances (N from {32, 40, 48, 64}, sigma ~
    U[1e6, 5e6] S/m, 100-1000 A, Brauer iron, SPE 8) advanced together with FP32 inner
    solves in FP64 refinement (every solve to the FP64 true residual 1e-10), the block
    scale tuned during the warm-up, then `args.batch_sub_steps` timed batch steps (device
    time from the fork of the batch streams to their join).  Beside it, the same instances
    in the plain single-instance FP64 form: each alone on the whole GPU, from rest, the
    same warm-up and the same timed steps (device time of each)."""
    import dataclasses
    import numpy as np
    import torch
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    probs = W.batched_instances(args.batch_sub, sizes=(32, 40, 48, 64))
    t0 = time.perf_counter()
    lam_ref = {}
    for n in sorted({p.N for p in probs}):
        s = pkg.Solver.from_problem(W.scaled_nonlinear(n), pkg.SolverOptions(tol=1e-10))
        lam_ref[n], _ = s.lambda_max(W.power_start_vector(s.n_c), pcg_tol=1e-12, rtol=1e-8, maxit=args.power_maxit)
        s.close()
    opts, solvers = [], []
    for p in probs:
        lam = lam_ref[p.N] * 2.0e6 / float(p.sigma_cell.max())       # M_c scales with sigma
        o = pkg.SolverOptions(tol=1e-10, start_mode=pkg.START_SPE, spe_depth=8, precision=1, pcg_variant=1,
                              dt=0.9 * 2.0 / lam, graph=1)
        opts.append(o)
        solvers.append(pkg.Solver.from_problem(p, o))
    setup_s = time.perf_counter() - t0
    trial = 1
    batch = pkg.Batch(solvers)
    scale = batch.tune(trial)                       # 8 x trial warm-up steps (4 scales, twice)
    by_work = batch.weighting()
    forms = batch.tune_pcg(args.tune_pcg_trials) if args.tune_pcg else [s_.pcg_form() for s_ in solvers]   # PCG kernel form per grid size
    form_by_n = {int(p.N): {"pcg_variant": int(v[0]), "tile_groups": int(v[1]), "halo_warps": int(v[2])}
                 for p, v in zip(probs, forms)}
    extra = max(args.batch_sub_warmup - 8 * trial, 0)
    if extra:
        batch.step(extra)
    warm = 8 * trial + extra
    rc, stats = batch.step(args.batch_sub_steps, allow_fail=True)
    ms = batch.last_ms()
    batch.close()
    its = np.array([[x.iterations for x in row] for row in stats], dtype=float)
    failed = int(sum(1 for row in stats for x in row if x.status != 0))
    value = len(solvers) * args.batch_sub_steps / (ms * 1e-3)
    stream = torch.cuda.Stream(device=dev)
    per_ms, its64 = [], []
    for sv, o in zip(solvers, opts):
        sv.set_options(dataclasses.replace(o, precision=0, pcg_variant=0))
        sv.set_state(np.zeros(sv.n_c), 0.0, 0)
        sv.reset_history()
        sv.set_stream(stream.cuda_stream)
        sv.step(warm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st64 = sv.step(args.batch_sub_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        per_ms.append(e0.elapsed_time(e1))
        its64.extend(x.iterations for x in st64)
        sv.set_stream(0)
        sv.close()
    single = len(solvers) * args.batch_sub_steps / (sum(per_ms) * 1e-3)
    sizes = {n: sum(1 for p in probs if p.N == n) for n in sorted({p.N for p in probs})}
    return {"value": value, "unit": "instance-steps/s", "instances": len(solvers), "count_per_N": sizes,
            "n_unknowns": int(sum(p_n for p_n in (sv.n_n for sv in solvers))),
            "steps": args.batch_sub_steps, "first_step": warm + 1, "ms": ms,
            "precision": "FP32 inner CG in FP64 refinement (FP64 true residual 1e-10 per solve)",
            "blocks_scale": scale, "block_shares": "unknowns x iterations" if by_work else "unknowns",
            "pcg_form_by_N": form_by_n,
            "inner_iters_per_step": float(its.mean()), "failed_steps": failed,
            "single_instance_fp64": {"value": single, "unit": "instance-steps/s",
                                     "iters_per_step": float(np.mean(its64)),
                                     "note": "each instance alone on the whole GPU, FP64 PCG, the same steps"},
            "speedup_vs_single_instance_fp64": value / single, "setup_s": setup_s}


def adjoint_fd_check(args, p, fresh):
    """Central differences of J (solves at tol 1e-12) against the adjoint gradient:
    random iron cells with a gradient of at least 1% of the largest, and the coil
    amplitude, at relative steps 1e-6 and 1e-4."""
    import numpy as np
    sc = fresh(1e-12)
    J12, g12, gI12, _ = sc.adjoint(args.steps)
    sc.close()
    sig = p.sigma_cell.reshape(-1)
    g = g12.reshape(-1)
    rng = np.random.default_rng(1611)
    # random iron cells among those whose gradient is at least 1% of the largest (smaller ones
    # fall below what a difference quotient of J resolves at this size)
    cand = np.flatnonzero((sig > 0) & (np.abs(g) >= 1e-2 * np.abs(g).max()))
    cells = rng.choice(cand, size=min(max(args.fd_params - 1, 0), cand.size), replace=False)
    fd_err = {}
    for h in (1e-6, 1e-4):
        errs = []
        for c in cells:
            vals = []
            for sgn in (1.0, -1.0):
                sp = sig.copy()
                sp[c] *= 1.0 + sgn * h
                sv = fresh(1e-12, p.with_(sigma_cell=sp.reshape(p.sigma_cell.shape)))
                vals.append(sv.loss(args.steps))
                sv.close()
            fd = (vals[0] - vals[1]) / (2.0 * h * sig[c])
            errs.append(abs(g[c] - fd) / abs(fd))
        vals = []
        for sgn in (1.0, -1.0):
            sv = fresh(1e-12, p.with_(amplitude=p.amplitude * (1.0 + sgn * h)))
            vals.append(sv.loss(args.steps))
            sv.close()
        fdI = (vals[0] - vals[1]) / (2.0 * h * p.amplitude)
        fd_err[f"h_rel={h:g}"] = {"max_rel_err_cells": max(errs) if errs else None,
                                  "median_rel_err_cells": float(np.median(errs)) if errs else None,
                                  "amplitude_rel_err": abs(gI12 - fdI) / abs(fdI)}
    return fd_err, cells


def run_adjoint(args):
    """Gradient of the eddy-current loss J = sum_m dt F_m^T M_c^-1 F_m over the steps of
    the 64^3 iron workload from rest (mqs_adjoint: forward steps recording the
    conductor trajectory, then the reverse sweep with one K_n solve per step), FP64.
    value = steps per second of forward + reverse; the forward steps alone are timed
    on a second handle.  The gradient is checked against central differences
    (relative step 1e-6, solves at tol 1e-12) on args.fd_params parameters:
    conductivities of random iron cells and the coil amplitude."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p = W.config_nonlinear_iron() if args.grid == 64 else W.scaled_nonlinear(args.grid)
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10))
    lam, _ = s.lambda_max(W.power_start_vector(s.n_c), pcg_tol=1e-12, rtol=1e-8, maxit=args.power_maxit)
    s_nc = s.n_c
    s.close()
    dt = 0.9 * 2.0 / lam
    stream = torch.cuda.Stream(device=dev)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), out

    mode = {"zero": pkg.START_ZERO, "prev": pkg.START_PREV, "spe": pkg.START_SPE, "pod": pkg.START_POD,
            "cspe": pkg.START_CSPE}[args.start]
    depth = args.depth if args.depth else {"spe": 8, "cspe": 16}.get(args.start, 20)
    sopts = dict(start_mode=mode, spe_depth=depth if args.start in ("spe", "cspe") else 8,
                 pod_snapshots=depth if args.start == "pod" else 20, dt=dt, cspe_period=args.cspe_period)

    def fresh(tol, problem=None):
        sv = pkg.Solver.from_problem(problem or p, pkg.SolverOptions(tol=tol, **sopts))
        sv.set_stream(stream.cuda_stream)
        return sv
    sf = fresh(1e-10)
    sf.adjoint(5)                                        # warm-up (allocations, first launches)
    sf.close()
    sf = fresh(1e-10)
    ms_fwd, _ = timed(lambda: sf.step(args.steps))
    sf.close()
    sa = fresh(1e-10)
    ms_adj, (J, gs, gI, info) = timed(lambda: sa.adjoint(args.steps))
    sa.close()
    ck = None
    if args.checkpoint > 0:
        sc = fresh(1e-10)
        ms_ck, (Jc, gsc, gIc, infoc) = timed(lambda: sc.adjoint(args.steps, args.checkpoint))
        sc.close()
        gf, gcf = gs.reshape(-1), gsc.reshape(-1)
        ck = {"every": args.checkpoint, "steps_per_s": args.steps / (ms_ck * 1e-3),
              "recompute_iterations": int(infoc.recompute_iterations),
              "adjoint_iterations": int(infoc.adjoint_iterations),
              "rel_diff_grad_sigma_vs_full": float(np.linalg.norm(gcf - gf) / np.linalg.norm(gf)),
              "rel_diff_J": abs(Jc - J) / abs(J), "rel_diff_grad_amplitude": abs(gIc - gI) / abs(gI),
              "trajectory_bytes": 8 * s_nc * ((args.steps + args.checkpoint - 1) // args.checkpoint + 1)
                                  + 16 * s_nc * args.checkpoint}
    fd_err, cells = {}, []
    if args.fd_params > 0:
        fd_err, cells = adjoint_fd_check(args, p, fresh)
    line = {"metric": "adjoint gradient of the eddy-current loss (forward + reverse sweep), steps/s",
            "value": args.steps / (ms_adj * 1e-3), "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms_adj / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(p), "grid": p.N, "start": "rest", "tol": 1e-10,
                       "start_vector": args.start + (str(depth) if args.start in ("spe", "pod") else "")
                                       + " (forward and adjoint solves)", "dt_s": dt,
                       "parameters": f"{int((p.sigma_cell > 0).sum())} cell conductivities + coil amplitude",
                       "trajectory": "conductor state and rate of every step kept on the device"
                                     f" ({16 * s_nc * args.steps} bytes)"},
            "forward_only_steps_per_s": args.steps / (ms_fwd * 1e-3),
            "reverse_cost_vs_forward": (ms_adj - ms_fwd) / ms_fwd,
            "objective_J": J, "grad_amplitude": gI,
            "pcg_iterations": {"forward": int(info.forward_iterations), "adjoint": int(info.adjoint_iterations)},
            "fd_check": {"tol": 1e-12, "cells": len(cells),
                         "cells_from": "random iron cells with |dJ/dsigma| >= 1% of the largest", **fd_err}}
    if ck:
        line["checkpointed"] = ck
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false",
                    help="skip the end-to-end host C ABI timing of the same steps")
    ap.add_argument("--power-maxit", type=int, default=2000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=40.0, help="seconds of timed oracle steps at most")
    ap.add_argument("--no-cpu-all-cores", dest="cpu_all_cores", action="store_false",
                    help="skip the all-core oracle throughput")
    ap.add_argument("--reference-budget", type=float, default=150.0)
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per PCG launch, if measured")
    ap.add_argument("--start", choices=["zero", "prev", "spe", "pod", "cspe"], default="spe",
                    help="start vector of each step's solve (default: SPE)")
    ap.add_argument("--depth", type=int, default=0,
                    help="SPE depth, CSPE column cap or POD snapshot count (default 8 / 16 / 20)")
    ap.add_argument("--cspe-period", type=int, default=0, help="CSPE: steps between freezes (default 25)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="0: FP64 PCG (default); 1: FP32 / 2: float-float inner solves in FP64 refinement "
                         "(same tolerance)")
    ap.add_argument("--eps-lin", type=float, default=1e-10,
                    help="SPE drop tolerance: a column is dropped when its K-remainder falls below eps_lin x the "
                         "newest solution's K-norm")
    ap.add_argument("--no-alt", dest="alt", action="store_false",
                    help="skip timing the FP32- and float-float-inner paths beside the FP64 line")
    ap.add_argument("--rhs-split", action="store_true",
                    help="solve the conductor-type and coil-type right-hand sides separately, each with its own "
                         "SPE history (the paper's separate right-hand sides)")
    ap.add_argument("--graph", type=int, default=1, choices=[0, 1],
                    help="replay steady-state SPE steps from CUDA graphs (1, default) or issue every launch (0)")
    ap.add_argument("--pcg-variant", type=int, default=1, choices=[0, 1, 2],
                    help="0: two grid reductions per PCG iteration, 1: one (fused pass; default), 2: with "
                         "--precision 1, the inner pass carrying x, r, p only (24 B per unknown)")
    ap.add_argument("--halo-warps", type=int, default=2, choices=[0, 1, 2],
                    help="one-reduction passes (FP64, and the FP32 inner pass below 96^3): halo warps per tile "
                         "group (0/1: one; 2: two, in 384-thread blocks, the default)")
    ap.add_argument("--grid", type=int, default=64,
                    help="cells per axis of the iron workload (64: the benchmark; others scale it)")
    ap.add_argument("--dt", type=float, default=0.0, help="time step in s (default: 0.9 * 2 / lambda_max)")
    ap.add_argument("--sweep", type=str, default="",
                    help="comma-separated grid sizes: time zero-start solves at each (roofline evidence)")
    ap.add_argument("--no-tune-pcg", dest="tune_pcg", action="store_false",
                    help="batched modes: keep --pcg-variant instead of the kernel-form tuner's choice per N")
    ap.add_argument("--tune-pcg-trials", type=int, default=3, help="timed trial solves per kernel form")
    ap.add_argument("--block-sweep", type=str, default="",
                    help="comma-separated grid sizes: PCG time per iteration against the block count")
    ap.add_argument("--batch-sub", type=int, default=64,
                    help="instances of the short batched measurement added to the line (0: skip)")
    ap.add_argument("--batch-sub-steps", type=int, default=20, help="timed steps of that batch")
    ap.add_argument("--batch-sub-warmup", type=int, default=16, help="its warm-up steps (tuning included)")
    ap.add_argument("--batch", type=int, default=0,
                    help="advance this many seeded multi-query instances together (batched mode)")
    ap.add_argument("--tune-depth", action="store_true",
                    help="batched mode: tune the SPE depth per grid size over {4, 8, 16} after the block scale")
    ap.add_argument("--batch-grid", type=str, default="",
                    help="comma-separated grid sizes the batched instances draw from (default 32,40,48,64)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the adjoint gradient of the eddy-current loss and check it by central differences")
    ap.add_argument("--fd-params", type=int, default=32, help="parameters checked by central differences")
    ap.add_argument("--checkpoint", type=int, default=25,
                    help="adjoint mode: also run with checkpoints every this many steps (0: skip)")
    ap.add_argument("--single-solve", action="store_true",
                    help="run one zero-start PCG solve of the workload twice (profiling)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=25.0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-warmup", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-dt", type=float, default=0.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_warmup, args.oracle_sample, args.oracle_budget, args.oracle_dt)),
              flush=True)
        return
    if args.single_solve:
        single_solve(args.pcg_variant, args.halo_warps)
        return
    if args.sweep:
        size_sweep([int(v) for v in args.sweep.split(",") if v])
        return
    if args.block_sweep:
        block_sweep([int(v) for v in args.block_sweep.split(",") if v])
        return
    if args.batch:
        run_batch(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("at least 3 warm-up steps")
    rank, ws, local, dist = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
    else:
        run_ours(args, rank, ws, local, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
