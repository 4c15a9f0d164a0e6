"""Oracle trajectories of the 4096-cell 14-moment Sod tube (at five
Knudsen numbers, RK2, MUSCL, minmod, HLL, CFL 0.5, to t = 0.2) for
tests/test_gpu_zsod14_4096.py.  They take minutes of CPU time, so conftest
starts them in a spawn-started process pool (OpenMP oracle, threads shared
out by the expected step counts) as soon as that test is collected, and the
rest of the GPU suite runs meanwhile.  Each run returns the final state, the
step sizes, and the states before and after a few sampled steps (for the
per-step parity gate)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, T_END = 4096, 0.2
# Kn -> OpenMP threads (longer runs get more; measured step counts to t = 0.2:
# 1e-3 12.5k, 1e-2 36k, 0.1 44k, 1 32k, 10 14.5k)
KN_THREADS = {0.1: 4, 0.01: 3, 1.0: 3, 10.0: 3, 0.001: 3}
SAMPLES = (0, 1, 1000, 5000, 10000, 20000, 30000, 40000)


def oracle_run(kn, threads):
    os.environ["OMP_NUM_THREADS"] = str(threads)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2401_15233_gb300 import workloads as wl
    cfg = oracle.make_cfg(system=14, nx=NX, ny=1, order=2, integrator=oracle.RK2,
                          tau_model=oracle.TAU_HARDSPHERE, tau_ref=wl.sod_tau_ref(kn))
    U = oracle.prim2cons_field(wl.sod_prim(14, NX)[None])
    t, k, dts, samples = 0.0, 0, [], {}
    while t < T_END:
        dt = oracle.dt(cfg, U, t, T_END, omp=True)
        if not dt > 0.0:
            break
        U1 = oracle.step(cfg, U, dt, omp=True)
        if k in SAMPLES:
            samples[k] = (U, dt, U1)
        U, t, k = U1, t + dt, k + 1
        dts.append(dt)
    return {"kn": kn, "U": U, "t": t, "steps": k, "dts": np.array(dts), "samples": samples}


class Runs:
    """The five oracle runs in a spawn-started pool (terminated on close)."""

    def __init__(self):
        import multiprocessing as mp
        if ROOT not in sys.path:
            sys.path.insert(0, ROOT)
        import oracle
        oracle.build(omp=True)                 # once, before the workers load it
        self.pool = mp.get_context("spawn").Pool(len(KN_THREADS), maxtasksperchild=1)
        self.res = {kn: self.pool.apply_async(oracle_run, (kn, th))
                    for kn, th in KN_THREADS.items()}

    def get(self, kn, timeout=3600):
        return self.res[kn].get(timeout)

    def close(self):
        self.pool.terminate()
        self.pool.join()
