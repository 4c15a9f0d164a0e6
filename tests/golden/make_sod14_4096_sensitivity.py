"""Writes sod14_4096_sensitivity.txt: the data sensitivity of the 4096-cell
14-moment Sod tube (RK2, MUSCL, minmod, HLL, CFL 0.5, hard-sphere BGK) at
t = 0.2 for Kn in {1e-3, 1e-2, 0.1, 1, 10}, computed by the FP64 oracle
alone: the relative L1 change of the density, the temperature
T = tr P / (3 rho) and the heat flux q_x when every primitive of the initial
state is perturbed by 1e-7 relative (random signs, seeded per Kn).  Ten
times these values is the bound of the mixed-precision path's L1 error
against the oracle (the mixed-precision accuracy reading).  Run from the
repository root:  python tests/golden/make_sod14_4096_sensitivity.py
(about twenty minutes on eight cores)."""
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
KNS = (1e-3, 1e-2, 0.1, 1.0, 10.0)
NX, T_END = 4096, 0.2


def fields(orc, U):
    """rho, T, q_x of conserved (1, nx, 14) states"""
    P = orc.cons2prim_field(U).reshape(-1, 14)
    rho = P[:, 0]
    return [rho, (P[:, 4] + P[:, 7] + P[:, 9]) / (3.0 * rho), P[:, 10]]


def run(args):
    kn, threads = args
    os.environ["OMP_NUM_THREADS"] = str(threads)
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2401_15233_gb300 import workloads as wl
    cfg = oracle.make_cfg(system=14, nx=NX, ny=1, order=2, integrator=oracle.RK2,
                          tau_model=oracle.TAU_HARDSPHERE, tau_ref=wl.sod_tau_ref(kn))
    prim = wl.sod_prim(14, NX)[None]
    rng = np.random.default_rng(int(round(1e6 * kn)))
    pert = prim * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=prim.shape))
    out = []
    for p in (prim, pert):
        U, t, hist = oracle.run(cfg, oracle.prim2cons_field(p), 0.0, T_END, 10 ** 7, omp=True)
        out.append((fields(oracle, U), t, len(hist)))
    (fa, ta, na), (fb, tb, nb) = out
    l1 = [float(np.abs(b - a).sum() / np.abs(a).sum()) for a, b in zip(fa, fb)]
    return kn, l1, na, nb


def main():
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build(omp=True)
    threads = max(1, (os.cpu_count() or 5) // len(KNS))
    with ProcessPoolExecutor(len(KNS), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(run, [(kn, threads) for kn in KNS]))
    lines = ["# Data sensitivity of the 14-moment Sod tube ( 4096 cells, RK2 MUSCL minmod HLL,",
             "# CFL 0.5, hard-sphere BGK, t = 0.2), FP64 oracle: relative L1 change of rho, T, q_x",
             "# under a 1e-7 relative perturbation of every initial primitive.",
             "# Written by make_sod14_4096_sensitivity.py (oracle only).  key = rho T q_x  (steps)"]
    for kn, l1, na, nb in res:
        lines.append(f"Kn{kn:g} = {l1[0]:.6e} {l1[1]:.6e} {l1[2]:.6e}  # {na} / {nb} steps")
    with open(os.path.join(HERE, "sod14_4096_sensitivity.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
