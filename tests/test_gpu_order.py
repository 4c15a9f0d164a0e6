"""Order of accuracy of the CUDA path on smooth data, and its agreement with
the oracle there (the shared limiter's flat-field test on the GPU):

  * the density wave at uniform velocity and pressure in the Euler limit
    (point-implicit BGK, tau = 1e-14, periodic) is advected by the FP64 path
    (5- and 14-moment) and the mixed path (14-moment) with an L1 error
    against the exact rho(x - u t) that falls at second order; before the
    flat-field test round-off in the uniform fields set the shared limiter
    to zero at random cells and the error fell at first order, ten times
    larger at 64 cells;
  * the FP64 path's free run to t = 0.1 lands on the oracle's free run (same
    step count, density within 1e-12): with noise-level differences no
    longer deciding the limiter, the two trajectories no longer separate.
"""
import numpy as np
import pytest

from tests._util import aos_to_soa
from tests.test_oracle_order import entropy_wave_prim

pytestmark = pytest.mark.gpu
T_END = 0.1


@pytest.fixture(scope="module")
def mx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as m
    m.lib()
    return m


def gpu_run(mx, system, n, precision, limiter):
    x = (np.arange(n) + 0.5) / n
    s = mx.Solver(system=system, nx=n, ny=1, order=2, integrator="rk2", precision=precision,
                  limiter=limiter)
    for side in (mx.XLO, mx.XHI):
        s.set_bc(side, mx.BC_PERIODIC)
    s.set_relaxation(mx.TAU_CONST, 1e-14)
    s.set_source_scheme("point_implicit")
    s.set_state(aos_to_soa(entropy_wave_prim(system, x)))
    t, steps = s.step(10 ** 6, T_END)
    assert t == pytest.approx(T_END, rel=1e-12)
    d = s.diagnostics()
    assert d["n_nonfinite"] == 0 and d["n_nonpositive"] == 0
    return s.get_moments("primitive")[:, 0, :], steps


def exact_density(n, t):
    x = (np.arange(n) + 0.5) / n
    h = 1.0 / n
    return 1 + 0.2 * (np.cos(2 * np.pi * (x - h / 2 - 0.5 * t))
                      - np.cos(2 * np.pi * (x + h / 2 - 0.5 * t))) / (2 * np.pi * h)


@pytest.mark.parametrize("system,precision,limiter", [(5, "fp64", "minmod"), (14, "fp64", "minmod"),
                                                      (14, "fp64", "vanalbada"),
                                                      (14, "mixed", "minmod"),
                                                      (14, "mixed", "vanalbada")])
def test_entropy_wave_second_order(mx, system, precision, limiter):
    e = []
    for n in (64, 128, 256, 512):
        Q, _ = gpu_run(mx, system, n, precision, limiter)
        assert np.abs(Q[1] - 0.5).max() < (1e-12 if precision == "fp64" else 1e-6)
        e.append(np.abs(Q[0] - exact_density(n, T_END)).mean())
    e = np.array(e)
    p = np.log2(e[:-1] / e[1:])
    print(f"system {system} {precision} {limiter}: L1 {e} orders {p}")
    assert e[0] < 2e-3 and np.all(p > 1.75), (e, p)


@pytest.mark.parametrize("system", [5, 14])
def test_entropy_wave_free_run_matches_oracle(mx, orc, system):
    n = 128
    Q, steps = gpu_run(mx, system, n, "fp64", "minmod")
    x = (np.arange(n) + 0.5) / n
    cfg = orc.make_cfg(system=system, nx=n, ny=1, order=2, integrator=1, tau_model=1,
                       tau_ref=1e-14, sides=[{"type": 1}] * 4,
                       source_scheme=orc.SRC_POINT_IMPLICIT)
    Uo, to, hist = orc.run(cfg, orc.prim2cons_field(entropy_wave_prim(system, x)), 0.0, T_END,
                           10 ** 6)
    Qo = orc.cons2prim_field(Uo)[0]
    diff = np.abs(Q[0] - Qo[:, 0]).max()
    print(f"system {system}: {steps} GPU steps, {len(hist)} oracle steps, max |rho diff| {diff:.2e}")
    assert steps == len(hist) and diff < 1e-12
