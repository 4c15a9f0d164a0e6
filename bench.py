#!/usr/bin/env python3
"""Throughput benchmark: 14-moment maximum-entropy crossed supersonic jets,
2D, midpoint RK2, MUSCL + shared minmod + HLL (Boccelli et al., JCP 2024),
on one GB300 per rank.

A step is one full RK2 step of the whole grid (two fused stage launches).
Metric: cell-updates/s (cells x steps / s).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 4096]
                  [--precision fp64|mixed] [--impl ours|reference]

The input (4096^2 x 14 fields x 8 B = 1.9 GB per state buffer) is far larger
than L2, so no flush is needed between timed steps.  N > 1 runs independent
replicas, one per GPU (the method is single-grid; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s 14-mom 2D RK2 (% HBM roofline), mixed vs FP64; adjoint/fwd ratio"
UNIT = "cell-updates/s"
# Algorithmic bytes per cell-update (one cell advanced one full RK2 step):
# each stage reads its inputs once and writes its output once, 14 fields.
#   fp64 : stage 1 reads U^n, writes U*; stage 2 reads U*, U^n, writes
#          U^{n+1}: 5 x 14 x 8 B = 560 B
#   mixed: U^n FP64 (the conservation accumulator), U* FP32: stage 1 reads
#          U^n (112), writes U* (56); stage 2 reads U* (56), U^n (112),
#          writes U^{n+1} (112): 448 B
# This is the roofline's basis.  The kernels move less for planar states
# (u_z, P_xz, P_yz, q_z identically zero, as in the crossed jets): ten
# fields, and the mixed path carries FP32 primitives W beside U^n:
#   fp64 planar 400 B; mixed planar: stage 1 reads W, writes Ws (2 x 40);
#   stage 2 reads Ws, U^n, W, writes U^{n+1}, W (3 x 40 + 2 x 80): 360 B
BYTES_PER_CELL_UPDATE = {"fp64": 560.0, "mixed": 448.0}
PLANAR_BYTES_PER_CELL_UPDATE = {"fp64": 400.0, "mixed": 360.0}
# DRAM bytes per cell-update measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over the two stage launches of step 1001 of the
# crossed jets from rest at 2048^2, 4.19e6 cells; scaled to the benchmark grid
# by cell count)
TRAFFIC_PER_CELL_UPDATE = {("mixed", True): 342.4}
# Issue-rate roofline of the mixed planar stage kernel (bound by instruction
# issue, not by DRAM): thread instructions per cell-update over both stages
# (ncu smsp__inst_executed.sum x 32 / cells, the same two launches) against
# 152 SMs x 4 schedulers x 32 lanes x the sampled SM clock.
THREAD_INST_PER_CELL_UPDATE = {("mixed", True): 5269.2}
KERNEL = {("fp64", False): "mxe_stage14_2d_f64", ("mixed", False): "mxe_stage14_2d_mixed_b3",
          ("fp64", True): "mxe_stage14_2d_f64_planar",
          ("mixed", True): "mxe_stage14_2d_mixed_planar_x2"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--prerun", type=int, default=1000,
                   help="untimed steps from the developed state before warm-up and timing")
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--compare-steps", type=int, default=10,
                   help="timed steps of the other precision")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--scalar-faces", action="store_true",
                   help="planar mixed stage: scalar face states instead of packed FP32 pairs")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched-tube leg (256 Sod tubes, one graph launch)")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the adjoint leg (512^2 crossed jets, 500 steps, checkpoints every 50)")
    p.add_argument("--no-jet", action="store_true",
                   help="skip the single collisionless jet leg (1200^2, forward Euler)")
    p.add_argument("--no-l1", action="store_true",
                   help="skip the per-field mixed-vs-FP64 L1 leg (1024^2, 200 steps)")
    p.add_argument("--no-dt-history", action="store_true",
                   help="skip the crossing collisionless jets step-size history (1200^2, 10000 steps)")
    p.add_argument("--cpu-full", action="store_true",
                   help="CPU baseline: also the 4096-cell 14-moment Sod tube to t = 0.2 and the crossed jets at 1024^2 for 20 steps")
    p.add_argument("--only", default=None, choices=["batch", "adjoint", "cpu", "l1", "dt"],
                   help="run one secondary leg alone (profiling runs)")
    p.add_argument("--batch-t-end", type=float, default=0.2)
    p.add_argument("--batch-shape", default=None,
                   help="block shape of the batched tubes as THREADSxCTAS (e.g. 256x8) "
                        "instead of the autotuner's choice")
    p.add_argument("--adj-n", type=int, default=512)
    p.add_argument("--adj-steps", type=int, default=500)
    p.add_argument("--adj-ckpt", type=int, default=50)
    p.add_argument("--adj-precision", default=None, choices=["fp64", "mixed"],
                   help="--only adjoint: one reverse precision, no finite differences")
    return p.parse_args()


def finite_json(x):
    """Non-finite floats -> null (strict JSON)."""
    if isinstance(x, float):
        return x if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: finite_json(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [finite_json(v) for v in x]
    return x


def issue_roofline(precision, planar, ncell, step_s, clk):
    """Achieved thread-instruction issue rate of one step of the stage
    kernel against the scheduler peak at the sampled SM clock."""
    per = THREAD_INST_PER_CELL_UPDATE.get((precision, planar))
    if per is None:
        return None
    mhz = (clk.summary() or {}).get("sm_mhz") if clk else None
    mhz = mhz or 2070.0
    peak = 152 * 4 * 32 * mhz * 1e6 / 1e12
    ach = per * ncell / step_s / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinst/s", "frac": ach / peak,
            "thread_inst_per_cell_update": per, "peak_from": "152 SMs x 4 x 32 lanes x sm_mhz"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms; only the
    samples whose timestamps fall inside the timed region (mark_start() ..
    mark_end()) are summarised."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None
        self._summary = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.5)
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        time.sleep(0.15)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self._summary is not None:
            return self._summary
        import datetime
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        n_all = 0
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    smv, mxv = float(f[2]), float(f[3])
                except ValueError:
                    continue
                n_all += 1
                if self.t0 is not None and not (self.t0 - 0.05 <= ts <= self.t1 + 0.05):
                    continue
                sm.append(smv); mx.append(mxv)
                for n, v in zip(names, f[6:10]):
                    if v.lower() == "active":
                        reasons.add(n)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        if not sm:
            self._summary = {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                             "samples_outside_region": n_all}
        else:
            self._summary = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                             "reasons": sorted(reasons), "samples": len(sm),
                             "timed_region_s": self.t1 - self.t0}
        return self._summary


def dist_setup(args, backend=None):
    """One process per GPU (torchrun env).  Replicas: the only collective is
    the max over ranks of the timed region."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend or "nccl")
    return world, rank, local, dist


def max_over_ranks(x, dist, device="cuda"):
    """max of a per-rank float over all ranks (identity without a group)"""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, total_ms):
    """throughput of all ranks' units over the slowest rank's time (weak scaling)"""
    return world * units_per_rank / (total_ms * 1e-3)


def make_solver(mx, wl, n, precision, setup):
    s = mx.Solver(system=14, nx=n, ny=n, precision=precision, order=2, integrator="rk2",
                  flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4)
    lo, hi = setup["slot"]
    s.set_bc(mx.XLO, mx.BC_DIRICHLET, lo, hi, setup["left"])
    s.set_bc(mx.YLO, mx.BC_DIRICHLET, lo, hi, setup["bottom"])
    s.set_relaxation(mx.TAU_HARDSPHERE, setup["tau_ref"], setup["rho_ref"], setup["T_ref"])
    return s


def cpu_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine()}


def _jets_oracle(oracle, wl, n, rest=False):
    """The crossed-jets workload on an n x n grid for the oracle: its
    configuration and the developed state, or (rest) the background at rest
    the run starts from (conserved, (n, n, 14))."""
    import numpy as np
    setup = wl.jets_setup(Kn=0.1)
    prim = wl.jets_initial(n, n, setup) if rest else wl.jets_like_field(n, n, setup)
    U = oracle.prim2cons_field(prim)
    lo, hi = setup["slot"]
    sides = [{"type": 0, "spans": [(lo, hi, setup["left"])]}, {"type": 0},
             {"type": 0, "spans": [(lo, hi, setup["bottom"])]}, {"type": 0}]
    cfg = oracle.make_cfg(system=14, nx=n, ny=n, tau_model=2, tau_ref=setup["tau_ref"],
                          rho_ref=setup["rho_ref"], T_ref=setup["T_ref"], sides=sides)
    return cfg, np.ascontiguousarray(U)


def _timed_steps(oracle, cfg, U, omp, seconds, max_steps):
    """RK2 steps of the oracle (CFL step included) until `seconds` or
    `max_steps`; returns (steps, elapsed seconds)."""
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        U = oracle.step(cfg, U, oracle.dt(cfg, U, 0.0, 10.0, omp=omp), omp=omp)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    return steps, time.perf_counter() - t0


def cpu_baseline(wl, full=False):
    """The FP64 oracle as it stands on the host cores: single-threaded (the
    paper's 1-core basis) and its OpenMP build on all cores (bitwise the
    same arithmetic), on bounded samples of the benchmark workloads: the
    crossed jets (RK2, MUSCL, HLL) on a 128^2 grid, the 5-moment Sod tube
    (1000 cells, first order, forward Euler) to t = 0.2 in full, the 14-moment
    Sod tube (4096 cells, RK2, Kn = 0.01) over its first 100 steps.  full: also
    the 14-moment tube to t = 0.2 and the crossed jets at 1024^2 for 20 steps
    (minutes of CPU time).  Rate = cell-updates/s."""
    import oracle
    oracle.build()
    oracle.build(omp=True)
    info = cpu_info()
    threads = oracle.threads(omp=True)
    out = {"kind": "oracle", "unit": UNIT, **info, "threads_all_core": threads}

    def leg(name, cells, run):
        r = {}
        for omp in (False, True):
            n, el = run(omp)
            r["all_core" if omp else "single_thread"] = {
                "value": cells * n / el, "steps": n, "seconds": el,
                "threads": threads if omp else 1}
        r["cells"] = cells
        out[name] = r

    def c3(n, seconds, max_steps):
        def run(omp):
            cfg, U = _jets_oracle(oracle, wl, n)
            return _timed_steps(oracle, cfg, U, omp, seconds, max_steps)
        return run

    def sod(system, nx, order, integ, t_end, max_steps):
        import numpy as np

        def run(omp):
            U = oracle.prim2cons_field(wl.sod_prim(system, nx)[None])
            cfg = oracle.make_cfg(system=system, nx=nx, ny=1, order=order, integrator=integ,
                                  tau_model=oracle.TAU_HARDSPHERE, tau_ref=wl.sod_tau_ref(0.01))
            t0 = time.perf_counter()
            _, _, hist = oracle.run(cfg, np.ascontiguousarray(U), 0.0, t_end, max_steps, omp=omp)
            return len(hist), time.perf_counter() - t0
        return run

    leg("jets_128", 128 * 128, c3(128, 8.0, 200))
    leg("sod5_1000_to_t0.2", 1000, sod(5, 1000, 1, oracle.FE, 0.2, 10 ** 6))
    leg("sod14_4096_100_steps", 4096, sod(14, 4096, 2, oracle.RK2, 0.2, 100))
    if full:
        leg("sod14_4096_to_t0.2", 4096, sod(14, 4096, 2, oracle.RK2, 0.2, 10 ** 7))
        leg("jets_1024_20_steps", 1024 * 1024, c3(1024, 1e9, 20))
    h = out["jets_128"]["all_core"]
    out["value"] = h["value"]
    out["cores"] = threads
    out["sample"] = (f"128x128 crossed jets (the benchmark workload's set-up), {h['steps']} RK2 "
                     f"steps incl. CFL, {h['seconds']:.1f} s, OpenMP build on {threads} threads; "
                     f"single-thread and the Sod tubes beside it")
    return out


def bench_mixed_l1(mx, wl, stream, n=1024, steps=200):
    """Per-field error of the mixed path against the all-FP64 GPU path
    (held to 1e-12 of the FP64 oracle by the parity tests), crossed jets from
    the developed state, same step sizes.  Bound (fixed before measuring):
    10x the relative L1 change of the FP64 path when every primitive of the
    initial and inflow states is perturbed by 1e-7 relative (the data
    resolution of FP32).  Fields: the 14 conserved moments (the gate of the
    tests), and the primitive density, velocity, temperature, heat flux."""
    import numpy as np
    setup = wl.jets_setup(Kn=0.1)
    rng = np.random.default_rng(n)
    prim = np.ascontiguousarray(np.moveaxis(wl.jets_like_field(n, n, setup), -1, 0))

    def run(precision, st, init, dts=None):
        s = make_solver(mx, wl, n, precision, st)
        s.set_stream(stream.cuda_stream)
        s.set_state(init)
        if dts is None:
            s.set_dt_history(steps)
            s.step(steps, float("inf"))
            dts = s.dt_history(steps)
        else:
            s.step_dt(dts)
        return s.get_moments("conserved"), s.get_moments("primitive"), dts

    A, Ap, dts = run("fp64", setup, prim)
    pert = lambda x: x * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=np.shape(x)))
    a = math.sqrt(wl.GAMMA_3D)
    r1, u1, T1 = pert(np.array([1.0, 3.0 * a, 1.0]))
    r2, u2, T2 = pert(np.array([1.0, 3.0 * a, 1.0]))
    setup_p = dict(setup, left=wl.maxwellian14(r1, u1, 0.0, T1),
                   bottom=wl.maxwellian14(r2, 0.0, u2, T2))
    B, Bp, _ = run("fp64", setup_p, pert(prim), dts)
    G, Gp, _ = run("mixed", setup, prim, dts)

    def l1(a, b):
        a = a.reshape(a.shape[0], -1); b = b.reshape(b.shape[0], -1)
        den = np.abs(b).sum(1)
        return np.abs(a - b).sum(1) / np.where(den > 0, den, 1.0)

    names = ["rho", "rho_ux", "rho_uy", "rho_uz", "Exx", "Exy", "Exz", "Eyy", "Eyz", "Ezz",
             "Hx", "Hy", "Hz", "E4"]
    e, sens = l1(G, A), l1(B, A)
    nz = np.abs(A).reshape(14, -1).sum(1) > 0
    bound = np.maximum(10 * sens, 1e-10)

    def derived(P):            # rho, u_x, u_y, T, q_x, q_y, R/(rho theta^2)
        rho = P[0]
        T = (P[4] + P[7] + P[9]) / (3 * rho)
        return np.stack([rho, P[1], P[2], T, P[10], P[11], P[13] / (rho * T * T)])

    dn = ["rho", "u_x", "u_y", "T", "q_x", "q_y", "R_star"]
    ed, sd = l1(derived(Gp), derived(Ap)), l1(derived(Bp), derived(Ap))
    return {
        "workload": f"crossed jets {n}x{n} from the developed state, {steps} RK2 steps "
                    f"(t = {float(dts.sum()):.3e}), mixed vs all-FP64 GPU path, same step sizes",
        "conserved": {nm: {"l1": float(e[k]), "bound": float(bound[k])}
                      for k, nm in enumerate(names) if nz[k]},
        "primitive": {nm: {"l1": float(ed[k]), "bound": float(max(10 * sd[k], 1e-10))}
                      for k, nm in enumerate(dn)},
        "max_l1_over_bound": float((e[nz] / bound[nz]).max()),
        "within_bound": bool(np.all(e[nz] <= bound[nz])),
    }


def bench_dt_history(mx, wl, stream, n=1200, steps=10000):
    """Sec. 6 crossing collisionless jets (Mach 5, width L/7, background 1e-5
    of the jet density, no collision source), 1200^2, MUSCL + forward Euler
    at CFL 0.5, mixed precision: the step-size history over `steps` steps
    (the paper reports the step size collapsing near step 9000 on its
    1200^2 grid).  Reports the step size at chosen steps, its minimum, and
    the first step whose size falls below a tenth (and a hundredth) of the
    size at step 100."""
    import numpy as np
    import torch
    setup = wl.collisionless_jets_setup(2)
    lo, hi = setup["slot"]
    bg = setup["background"]
    s = mx.Solver(system=14, nx=n, ny=n, precision="mixed", order=2, integrator="fe",
                  flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4)
    s.set_stream(stream.cuda_stream)
    for side in (mx.XLO, mx.XHI, mx.YLO, mx.YHI):
        s.set_bc(side, mx.BC_DIRICHLET, 0.0, 0.0, bg)
    s.set_bc(mx.XLO, mx.BC_DIRICHLET, lo, hi, setup["left"])
    s.set_bc(mx.YLO, mx.BC_DIRICHLET, lo, hi, setup["bottom"])
    s.set_state(np.ascontiguousarray(np.moveaxis(wl.jets_initial(n, n, setup), -1, 0)))
    s.set_dt_history(steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stop = None
    try:                       # stops early if the step size collapses to zero
        s.step(steps, float("inf"))
    except mx.MaxentError as e:
        stop = str(e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    d = s.diagnostics()
    taken = int(d["steps"])
    dts = s.dt_history(taken)
    ref = float(dts[100]) if taken > 100 else float(dts[0])

    def first_below(f):
        k = np.nonzero(dts < f * ref)[0]
        return int(k[0]) if k.size else None

    marks = [k for k in (0, 100, 1000, 2000, 3000, 4000, 5000, 6000, 7000, 8000, 9000, 10000)
             if k < taken] + [taken - 1]
    return {"workload": f"two crossing collisionless jets {n}x{n}, Mach 5, FE MUSCL HLL minmod, "
                        f"CFL 0.5, mixed, up to {steps} steps",
            "steps_taken": taken, "stopped": stop,
            "dt_at_step": {str(k): float(dts[k]) for k in marks}, "dt_min": float(dts.min()),
            "step_of_dt_min": int(np.argmin(dts)), "t_final": float(dts.sum()),
            "first_step_dt_below_0.1_of_step100": first_below(0.1),
            "first_step_dt_below_0.01_of_step100": first_below(0.01),
            "ms_per_step": ms / max(taken, 1), "n_nonfinite": d["n_nonfinite"],
            "n_nonpositive": d["n_nonpositive"], "n_sigma_above_one": d["n_sigma_above_one"],
            "n_sigma_below_lim": d["n_sigma_below_lim"],
            "fp64_closure_share": (d["n_fp64_closures"] / d["n_closures"])
            if d["n_closures"] else None}


def bench_batch(mx, wl, stream, world, t_end=0.2, shape=None):
    """Batched 14-moment Sod tubes: 256 tubes of 512..8192 cells, Kn in
    [1e-3, 10], density ratio in [4, 20], each run to t = 0.2 in one persistent
    launch replayed from a CUDA graph, block shape from the autotuner.  Also
    times the FP64 batch (one block per tube) against the mixed batch over the
    first 20 steps of every tube, from the same initial state."""
    import numpy as np
    import torch
    tubes = wl.batch_tubes()
    ncells = np.array([t[0] for t in tubes], dtype=np.int64)
    prims = [np.ascontiguousarray(np.moveaxis(wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r), -1, 0))
             for (nc, kn, r) in tubes]

    def make(prec):
        b = mx.Batch(list(ncells), [1.0] * len(tubes), system=14, precision=prec, order=2,
                     integrator="rk2", flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4)
        b.set_stream(stream.cuda_stream)
        b.set_state(b.pack(prims))
        for i, (nc, kn, r) in enumerate(tubes):
            b.set_tube_relaxation(i, mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
        return b

    def timed_run(b, t_end, max_steps=10 ** 8):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.run(max_steps, t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        t, st = b.clock()
        return e0.elapsed_time(e1), int((ncells * st).sum()), st

    b = make("mixed")
    if shape:
        nt, cl = (int(x) for x in shape.lower().split("x"))
        b.set_shape(nt, cl)
        tune_ms = None
    else:
        nt, cl, tune_ms = b.autotune(0.002)
    b.run(10 ** 8, t_end)                 # warm-up: captures the graph for t_end
    b.set_state(b.pack(prims))            # back to t = 0 (same launch arguments: replay)
    ms, cu, st = timed_run(b, t_end)
    d = b.diagnostics()
    teams, team_tubes, fill = b.layout()
    bw = make("mixed")
    bw.set_shape(nt, cl)
    bw.run(20, 0.2)
    bw.set_state(b.pack(prims))
    ms_w, cu_w, _ = timed_run(bw, 0.2, 20)
    del bw
    bf = make("fp64")
    bf.run(3, 0.2)
    bf.set_state(b.pack(prims))
    ms_f, cu_f, _ = timed_run(bf, 0.2, 20)
    del bf
    return {
        "workload": "batched 14-moment Sod: 256 tubes, 512..8192 cells (log-uniform, seed "
                    "20240127), Kn 1e-3..10, density ratio 4..20, RK2 MUSCL minmod HLL, to t = 0.2",
        "precision": "mixed", "value": world * cu / (ms * 1e-3), "unit": UNIT,
        "ms": ms, "cell_updates": cu, "cells": int(ncells.sum()),
        "steps_min": int(st.min()), "steps_max": int(st.max()),
        # the timed run: one graph replay (queue reset, team launch, fill launch)
        "graph_launches": 1, "gpu_launches": 2 if fill else 1,
        "layout": {"teams": teams, "team_tubes": team_tubes, "fill_ctas": fill,
                   "fill_tubes": len(tubes) - team_tubes},
        "shape": {"threads_per_cta": nt, "ctas_per_team": cl, "autotune_ms_t0.002": tune_ms},
        "fp64_closure_share": (d["n_fp64_closures"] / d["n_closures"]) if d["n_closures"] else None,
        "n_nonfinite": d["n_nonfinite"], "n_nonpositive": d["n_nonpositive"],
        "first_20_steps": {"mixed": world * cu_w / (ms_w * 1e-3),
                           "fp64": world * cu_f / (ms_f * 1e-3),
                           "speedup": (cu_w / ms_w) / (cu_f / ms_f), "unit": UNIT},
    }


def bench_single_jet(mx, wl, stream, world, n=1200):
    """Sec. 6 single collisionless jet (Mach 5, width L/7, background 1e-5,
    no collision source), 1200^2, MUSCL + forward Euler, CFL 0.5, from the
    background: cell-updates/s of the mixed and the FP64 paths (steps 5..25
    and 5..15), and the step sizes seen."""
    import numpy as np
    import torch
    setup = wl.collisionless_jets_setup(1)
    lo, hi = setup["slot"]
    prim = np.ascontiguousarray(np.moveaxis(wl.jets_initial(n, n, setup), -1, 0))
    out = {"workload": f"single collisionless jet {n}x{n}, Mach 5, FE MUSCL HLL minmod, CFL 0.5"}
    for prec, steps in (("mixed", 20), ("fp64", 10)):
        s = mx.Solver(system=14, nx=n, ny=n, precision=prec, order=2, integrator="fe",
                      flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4)
        s.set_stream(stream.cuda_stream)
        for side in (mx.XLO, mx.XHI, mx.YLO, mx.YHI):
            s.set_bc(side, mx.BC_DIRICHLET, 0.0, 0.0, setup["background"])
        s.set_bc(mx.XLO, mx.BC_DIRICHLET, lo, hi, setup["left"])
        s.set_state(prim)
        s.set_dt_history(5 + steps)
        s.step(5, float("inf"), sync=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps, float("inf"), sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        dts = s.dt_history(5 + steps)
        out[prec] = {"value": whole_job_value(n * n * steps, world, ms), "unit": UNIT,
                     "ms_per_step": ms / steps, "dt_first": float(dts[0]), "dt_last": float(dts[-1])}
        del s
    out["speedup"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def bench_adjoint(world, n=512, nsteps=500, ckpt=50, only_precision=None):
    """Discrete adjoint of the crossed jets, 512^2, Kn = 0.1, 500 RK2 steps
    from the background at rest: gradient of the mean density over a 32 x 32
    probe w.r.t. both Mach numbers and tau_ref.  Cost ratio = (forward
    keeping what the backward needs + backward) / plain forward, host wall
    time around device-synchronised work, for the FP64 reverse and the FP32
    face-state reverse, with the configured checkpoints every 50 steps
    (each segment replayed before its sweep) and with the whole tape kept in
    device memory (recorded by the forward march, 2 x 500 states of 29 MB).
    Gradients beside central differences of the frozen-dt map (h = 1e-4 on
    the Mach numbers, 1e-4 relative on tau_ref):
      - the configured probe at the jet intersection: 500 steps carry
        signals ~0.1 of the domain, so the probe is outside the inflows'
        domain of dependence and both sides are zero;
      - the probe on the left inflow slot with first-order reconstruction
        (a smooth map): the non-zero check.  With MUSCL the shared limiter
        makes the map non-differentiable at the scale of any difference
        (checked instead against the oracle's tangent in the tests)."""
    import numpy as np
    import torch
    from paper_2401_15233_gb300 import adjoint as ad
    out = {"workload": f"crossed jets {n}x{n}, Kn 0.1, {nsteps} RK2 steps from rest; FP64 forward"}
    first_use = {}
    for prec in ("fp64", "mixed"):          # one-time costs of each reverse, outside the timing
        w = ad.JetsProblem(n=64, nsteps=20, ckpt=10, probe=8, initial="rest",
                           adjoint_precision=prec, tape="recompute")
        t0 = time.perf_counter()
        Jw, c, d, sw = ad.forward_checkpointed(w, w.params0())
        ad.backward_checkpointed(w, sw, c, d)
        torch.cuda.synchronize()
        first_use[prec] = time.perf_counter() - t0
        del sw, c
    out["first_use_64sq_s"] = first_use

    def timed_case(prob, legs):
        p0 = prob.params0()
        s = prob.solver(p0)
        s.set_state(prob.initial())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(prob.nsteps, float("inf"))
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        del s
        res = {"forward_s": tf}
        for prec, tape in legs:
            prob.adjoint_precision, prob.tape = prec, tape
            t0 = time.perf_counter()
            J, ckpts, dts, s2 = ad.forward_checkpointed(prob, p0)
            torch.cuda.synchronize()
            tfc = time.perf_counter() - t0
            t0 = time.perf_counter()
            g, _ = ad.backward_checkpointed(prob, s2, ckpts, dts)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            res[f"{prec}_{tape}"] = {"forward_keep_s": tfc, "backward_s": tb,
                                     "ratio": (tfc + tb) / tf, "grad": [float(x) for x in g],
                                     "fp64_fallback_segments": prob.fp64_fallbacks}
            del s2, ckpts
        fd = []
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-4 * (p0[2] if k == 2 else 1.0)
            fd.append((ad.run_fixed(prob, p0 + e, dts) - ad.run_fixed(prob, p0 - e, dts)) / (2 * e[k]))
        res.update({"J": J, "t_final": float(dts.sum()), "fd": [float(x) for x in fd]})
        return res

    legs = [(only_precision, "recompute")] if only_precision else [
        ("fp64", "recompute"), ("mixed", "recompute"), ("fp64", "keep"), ("mixed", "keep")]
    prob = ad.JetsProblem(n=n, nsteps=nsteps, ckpt=ckpt, probe=32, initial="rest", order=2)
    conf = timed_case(prob, legs)
    conf["probe"] = "32x32 at the jet intersection (0.5, 0.5), MUSCL"
    conf["probe_at_background"] = bool(conf["J"] == prob.setup["background"][0])
    out["configured"] = conf
    if only_precision:
        return out
    out["ratio"] = conf["fp64_recompute"]["ratio"]
    out["ratio_fp64_tape_kept"] = conf["fp64_keep"]["ratio"]
    out["ratio_fp32_reverse"] = conf["mixed_recompute"]["ratio"]
    slot = ad.JetsProblem(n=n, nsteps=nsteps, ckpt=ckpt, probe=32, initial="rest", order=1,
                          probe_at="left_slot")
    sl = timed_case(slot, [("fp64", "keep"), ("mixed", "keep")])
    sl["probe"] = "32x32 on the left inflow slot, first-order reconstruction"
    fd = np.array(sl["fd"])
    nz = np.abs(fd) > 0
    for key in ("fp64_keep", "mixed_keep"):
        g = np.array(sl[key]["grad"])
        sl[key]["max_rel_err_vs_fd_nonzero"] = float((np.abs(g[nz] - fd[nz]) / np.abs(fd[nz])).max())
        sl[key]["zero_components_exact"] = bool(np.all(g[~nz] == 0.0))
    out["slot_probe_first_order"] = sl
    return out


def workload_config(n, world, planar=True, prerun=0):
    """The benchmark's workload, as named in both arms' JSON lines (the
    arithmetic each arm computes in is its `dtype`)."""
    return {"workload": f"crossed supersonic jets, 14-moment 2D RK2, {n}x{n}",
            "n": n, "flux": "hll", "limiter": "minmod",
            "Kn": 0.1, "mach": 3, "parallelism": f"replicas{world}", "planar": planar,
            "initial": f"background at rest, jets from the slots; timed after {prerun} untimed steps",
            "l2": "inputs larger than L2 (1.9 GB per state buffer), no flush"}


def run_reference(args, wl):
    """The reference arm: the FP64 oracle on the host cores (its OpenMP
    build, bitwise the arithmetic of the single-threaded oracle), each step
    one RK2 step (CFL included) of a bounded 96^2 sample of the crossed-jets
    workload, run like the GPU arm's: from the background at rest, timed
    after the same number of untimed steps; rank 0 only."""
    world, rank, local, dist = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build(omp=True)
    threads = oracle.threads(omp=True)
    n = 96
    cfg, U = _jets_oracle(oracle, wl, n, rest=True)
    for _ in range(args.prerun + args.warmup):
        U = oracle.step(cfg, U, oracle.dt(cfg, U, 0.0, 10.0, omp=True), omp=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = oracle.step(cfg, U, oracle.dt(cfg, U, 0.0, 10.0, omp=True), omp=True)
    el = time.perf_counter() - t0
    v = n * n * args.steps / el
    info = cpu_info()
    sample = (f"{n}x{n} crossed jets per step (bounded sample of the {args.n}^2 workload), "
              f"from rest, timed after {args.prerun + args.warmup} untimed steps, "
              f"OpenMP oracle on {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.n, args.gpus, True, args.prerun),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, **info},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    from paper_2401_15233_gb300 import workloads as wl
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if args.only == "cpu":              # host cores only
        print(json.dumps(finite_json({"only": "cpu", "cpu": cpu_baseline(wl, args.cpu_full)})),
              flush=True)
        return
    import numpy as np
    import torch
    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_2401_15233_gb300 as mx
    if args.only:
        stream = torch.cuda.Stream()
        if args.only == "batch":
            leg = bench_batch(mx, wl, stream, world, args.batch_t_end, args.batch_shape)
        elif args.only == "cpu":
            leg = cpu_baseline(wl, args.cpu_full)
        elif args.only == "l1":
            leg = bench_mixed_l1(mx, wl, stream)
        elif args.only == "dt":
            leg = bench_dt_history(mx, wl, stream)
        else:
            leg = bench_adjoint(world, args.adj_n, args.adj_steps, args.adj_ckpt,
                                args.adj_precision)
        if rank == 0:
            print(json.dumps(finite_json({"only": args.only, args.only: leg})), flush=True)
        return

    n = args.n
    setup = wl.jets_setup(Kn=0.1)
    # the crossed-jets run: background at rest, jets entering through the slots
    # (the timed steps follow args.prerun untimed ones); the synthetic
    # developed state (a filled domain) is timed beside it
    rest = np.ascontiguousarray(np.moveaxis(wl.jets_initial(n, n, setup), -1, 0))
    developed = np.ascontiguousarray(np.moveaxis(wl.jets_like_field(n, n, setup), -1, 0))
    prim = rest
    ncell = n * n
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(precision, steps, sample_clocks, prerun=0, init=None):
        s = make_solver(mx, wl, n, precision, setup)
        s.set_stream(stream.cuda_stream)
        if precision == "mixed" and args.scalar_faces:
            s.set_face_packing(False)
        s.set_state(prim if init is None else init)
        if prerun:                  # untimed steps of the run first
            s.step(prerun, float("inf"))
        for _ in range(args.warmup):
            s.step(1, float("inf"), sync=False)
        barrier()
        s.diag0 = s.diagnostics()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.__enter__()
        barrier()
        if sampler:
            sampler.mark_start()
        ev[0].record(stream)
        for k in range(steps):
            s.step(1, float("inf"), sync=False)
            ev[k + 1].record(stream)
        barrier()
        if sampler:
            sampler.mark_end()
            sampler.__exit__()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        total_ms = max_over_ranks(total_ms, dist)
        # every timed step must have advanced the solution: a step whose
        # CFL size collapsed to zero does no work and would inflate the rate
        d1 = s.diagnostics()
        if d1["steps"] - s.diag0["steps"] != steps or d1["n_nonpositive"] or d1["n_nonfinite"]:
            raise RuntimeError(f"timed {precision} steps did not all advance: "
                               f"{d1['steps'] - s.diag0['steps']} of {steps}, "
                               f"non-positive cells {d1['n_nonpositive']}, "
                               f"non-finite {d1['n_nonfinite']}")
        return s, per, total_ms, sampler

    s, per, total_ms, clk = timed(args.precision, args.steps, True, args.prerun)
    d = s.diagnostics()
    d0 = s.diag0
    planar = bool(d["planar"])
    n_cl = d["n_closures"] - d0["n_closures"]
    fp64_share = (d["n_fp64_closures"] - d0["n_fp64_closures"]) / n_cl if n_cl else None
    value = whole_job_value(ncell * args.steps, world, total_ms)
    # the same kernels on the synthetic developed state (every cell in the
    # jets' non-equilibrium mix), first steps, no pre-run
    dsteps = max(10, min(args.steps, 20))
    sd, perd, totd, _ = timed(args.precision, dsteps, False, 0, developed)
    dd1, dd0 = sd.diagnostics(), sd.diag0
    ncd = dd1["n_closures"] - dd0["n_closures"]
    developed_leg = {"value": whole_job_value(ncell * dsteps, world, totd), "unit": UNIT,
                     "steps": dsteps, "ms_per_step": totd / dsteps,
                     "fp64_closure_share": ((dd1["n_fp64_closures"] - dd0["n_fp64_closures"]) / ncd
                                            if ncd else None)}
    del sd
    other = "fp64" if args.precision == "mixed" else "mixed"
    csteps = args.compare_steps or args.steps
    s2, per2, total2, _ = timed(other, csteps, False)
    other_value = whole_job_value(ncell * csteps, world, total2)
    planar2 = bool(s2.diagnostics()["planar"])
    del s2

    # end to end through the C-ABI with host buffers: H2D of the state,
    # one step, D2H of the state, every step.  The upload restores the state
    # the solver produced (kind "restore": the same validating copy kernel,
    # the realizability check reported but not enforced, because the scheme
    # may leave cells marginally outside sigma <= 1)
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(s.get_moments("conserved")).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        ne = max(2, min(args.steps, 10))
        s.set_state(host_in.numpy(), kind="restore")          # warm-up: a whole e2e step
        s.step(1, float("inf"), sync=False)
        s.get_moments("conserved", out=host_out.numpy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne):
            s.set_state(host_in.numpy(), kind="restore")
            s.step(1, float("inf"), sync=False)
            s.get_moments("conserved", out=host_out.numpy())
        el = time.perf_counter() - t0
        nbytes = host_in.numel() * 8
        e2e = {"value": world * ncell * ne / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ne}

    if rank != 0:
        return
    hbm, src = peaks()
    bpc = BYTES_PER_CELL_UPDATE[args.precision]
    kt = statistics.mean(per) * 1e-3        # one step = both stage launches of the kernel
    achieved = bpc * ncell / kt / 1e9
    bpc_p = PLANAR_BYTES_PER_CELL_UPDATE[args.precision] if planar else bpc
    bpc2 = BYTES_PER_CELL_UPDATE[other]
    ach2 = bpc2 * ncell / (statistics.mean(per2) * 1e-3) / 1e9
    traffic = TRAFFIC_PER_CELL_UPDATE.get((args.precision, planar))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 (+f64 accumulator, f64 closure islands)",
        "data": "synthetic",
        "config": workload_config(n, world, planar, args.prerun),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": traffic * ncell if traffic else None,
                     "kernel": KERNEL[(args.precision, planar)], "peak_source": src,
                     "bytes_per_cell_update": bpc,
                     "planar_basis": {"bytes_per_cell_update": bpc_p,
                                      "achieved": bpc_p * ncell / kt / 1e9,
                                      "frac": bpc_p * ncell / kt / 1e9 / hbm}},
        "roofline_issue": issue_roofline(args.precision, planar, ncell, kt, clk),
        "compare": {"precision": other, "value": other_value, "unit": UNIT, "steps": csteps,
                    "ms_per_step": total2 / csteps, "speedup_of_headline": value / other_value,
                    "roofline": {"bound": "hbm", "achieved": ach2, "peak": hbm, "unit": "GB/s",
                                 "frac": ach2 / hbm, "kernel": KERNEL[(other, planar2)],
                                 "bytes_per_cell_update": bpc2}},
        "gpu_launches": 2 * args.steps,
        "e2e": e2e,
        "clocks": clk.summary(),
        "diag": {"t": d["t"], "steps": d["steps"], "min_sigma": d["min_sigma"],
                 "n_sigma_below_lim": d["n_sigma_below_lim"], "n_nonfinite": d["n_nonfinite"],
                 "n_nonpositive": d["n_nonpositive"], "timed_steps_from": d0["steps"] + 1,
                 "fp64_closure_share_timed": fp64_share},
        "developed_state": developed_leg,
    }
    if not args.no_batch:
        out["batch"] = bench_batch(mx, wl, stream, world, args.batch_t_end, args.batch_shape)
    if not args.no_adjoint:
        out["adjoint"] = bench_adjoint(world)
    if not args.no_jet:
        out["single_jet"] = bench_single_jet(mx, wl, stream, world)
    if not args.no_l1:
        out["mixed_l1_per_field"] = bench_mixed_l1(mx, wl, stream)
    if not args.no_dt_history:
        out["crossing_jets_dt"] = bench_dt_history(mx, wl, stream)
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_full)
    print(json.dumps(finite_json(out)), flush=True)


if __name__ == "__main__":
    main()
