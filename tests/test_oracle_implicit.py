"""Pins of the oracle's point-implicit BGK source (backward-Euler relaxation
after each explicit stage; the remark closing Sec. 4.3 that a simple
point-implicit treatment suffices once the source limits the step):

  * a uniform state relaxes towards the Maxwellian built from its own
    density, velocity and temperature, whose moments come here from
    Gauss-Hermite quadrature (not from the oracle), by the backward-Euler
    factor 1 / (1 + dt/tau) per step, for both systems and both integrators;
  * in the stiff limit one step returns that Maxwellian, mass and momentum
    untouched;
  * mass and momentum are conserved to round-off under periodic BCs;
  * far from stiffness the implicit step differs from the explicit one by
    O(dt^2) (the local difference shrinks fourfold when dt halves);
  * Sod at Kn = 1e-5, where the explicit source is unstable at the CFL step,
    stays realizable with the implicit source and lands closer to the exact
    Euler Riemann solution than the explicit scheme does at Kn = 1e-3."""
import math

import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests.test_oracle_pins import psi5, psi14
from tests.test_oracle_scheme import exact_riemann

pytestmark = pytest.mark.filterwarnings("ignore")


def cons_field(orc, prim):
    return orc.prim2cons_field(prim)


def maxwellian_moments(system, Q):
    """Conserved moments of the Maxwellian with Q's density, velocity and
    temperature, by Gauss-Hermite quadrature (exact for these polynomials)."""
    from numpy.polynomial.hermite_e import hermegauss
    x, wq = hermegauss(6)
    wq = wq / math.sqrt(2 * math.pi)
    if system == 5:
        T = Q[2] / Q[0]
        v = x * math.sqrt(T) + Q[1]
        return (Q[0] * wq[:, None] * psi5(v)).sum(0)
    T = (Q[4] + Q[7] + Q[9]) / (3 * Q[0])
    V = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3) * math.sqrt(T) + Q[1:4]
    W = np.einsum("a,b,c->abc", wq, wq, wq).reshape(-1) * Q[0]
    return (W[:, None] * psi14(V)).sum(0)


def random_state(system, rng):
    if system == 14:
        return wl.random_prim14(rng, 1)[0]
    rho, u, P = 1.3, 0.4, 0.9
    return np.array([rho, u, P, 0.2, 3 * P * P / rho * 1.4])


def uniform_cfg(orc, system, tau, integ, scheme, n=4):
    return orc.make_cfg(system=system, nx=n, ny=1 if system == 5 else n, tau_model=1,
                        tau_ref=tau, integrator=integ, sides=[{"type": 1}] * 4,
                        source_scheme=scheme)


@pytest.mark.parametrize("system", [5, 14])
@pytest.mark.parametrize("integ", [0, 1])
def test_homogeneous_backward_euler_factor(orc, system, integ):
    rng = np.random.default_rng(31 + system)
    Q = random_state(system, rng)
    tau, dt, n = 0.3, 0.2, 7                      # dt/tau = 2/3: not small
    cfg = uniform_cfg(orc, system, tau, integ, orc.SRC_POINT_IMPLICIT)
    shape = (1, 4, system) if system == 5 else (4, 4, 14)
    U = np.broadcast_to(orc.prim2cons(Q), shape).copy()
    UM = maxwellian_moments(system, Q)
    d0 = U.reshape(-1, system)[0] - UM
    for _ in range(n):
        U = orc.step(cfg, U, dt)
    g = 1.0 / (1.0 + dt / tau)
    got = U.reshape(-1, system)[0] - UM
    np.testing.assert_allclose(got, g ** n * d0, rtol=1e-9, atol=1e-11 * np.abs(UM).max())


@pytest.mark.parametrize("system", [5, 14])
def test_stiff_limit_returns_the_maxwellian(orc, system):
    rng = np.random.default_rng(7)
    Q = random_state(system, rng)
    cfg = uniform_cfg(orc, system, 1e-14, 1, orc.SRC_POINT_IMPLICIT)
    shape = (1, 4, system) if system == 5 else (4, 4, 14)
    U0 = np.broadcast_to(orc.prim2cons(Q), shape).copy()
    U = orc.step(cfg, U0, 1e-3)
    UM = maxwellian_moments(system, Q)
    np.testing.assert_allclose(U.reshape(-1, system)[0], UM, rtol=1e-10,
                               atol=1e-12 * np.abs(UM).max())
    inv = 2 if system == 5 else 4
    assert np.array_equal(U[..., :inv], U0[..., :inv])


def test_conservation_periodic_2d(orc):
    n = 24
    rng = np.random.default_rng(9)
    prim = wl.smooth_field14(rng, n, n, amp=0.4)
    U = cons_field(orc, prim)
    cfg = orc.make_cfg(system=14, nx=n, ny=n, tau_model=2, tau_ref=1e-4,
                       sides=[{"type": 1}] * 4, source_scheme=orc.SRC_POINT_IMPLICIT)
    s0 = U.reshape(-1, 14).sum(0)
    e0 = s0[4] + s0[7] + s0[9]
    for _ in range(20):
        U = orc.step(cfg, U, orc.dt(cfg, U, 0.0, 10.0))
    s1 = U.reshape(-1, 14).sum(0)
    e1 = s1[4] + s1[7] + s1[9]
    scale = np.abs(U.reshape(-1, 14)).sum(0)
    assert np.all(np.abs(s1[:4] - s0[:4]) <= 1e-13 * scale[:4])
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    # and the non-equilibrium moments have relaxed (tau << dt)
    Q = orc.cons2prim_field(U).reshape(-1, 14)
    p = (Q[:, 4] + Q[:, 7] + Q[:, 9]) / 3
    assert np.abs(Q[:, 5]).max() < 1e-2 * p.max()


@pytest.mark.parametrize("system,integ", [(5, 0), (14, 0), (5, 1), (14, 1)])
def test_weak_relaxation_second_order_close_to_explicit(orc, system, integ):
    """Far from stiffness (dt/tau ~ 1e-3) one implicit step and one explicit
    step from the same Sod state differ by O(dt^2): the difference shrinks
    fourfold when dt halves.  First order in space (the shared MUSCL limiter
    of noise-level non-equilibrium differences is not a smooth function of
    the state and would hide the order)."""
    nx = 64
    U = cons_field(orc, wl.sod_prim(system, nx)[None])
    diffs = []
    for dt in (4e-5, 2e-5, 1e-5):
        out = []
        for scheme in (orc.SRC_EXPLICIT, orc.SRC_POINT_IMPLICIT):
            cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=1, integrator=integ,
                               tau_model=1, tau_ref=0.02, source_scheme=scheme)
            out.append(orc.step(cfg, U, dt))
        diffs.append(np.abs(out[1] - out[0]).max())
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    print(system, integ, diffs, r1, r2)
    assert diffs[-1] > 0
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6


@pytest.mark.parametrize("system,gam", [(5, 3.0), (14, 5.0 / 3.0)])
def test_euler_limit_with_point_implicit_source(orc, system, gam):
    nx, tend = 160, 0.15
    x = (np.arange(nx) + 0.5) / nx
    ex = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gam, (x - 0.5) / tend)
    U0 = cons_field(orc, wl.sod_prim(system, nx)[None])

    def run(Kn, scheme, max_steps=200000):
        cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=2, integrator=1, tau_model=2,
                           tau_ref=wl.sod_tau_ref(Kn), source_scheme=scheme)
        return orc.run(cfg, U0, 0.0, tend, max_steps)

    # explicit source at Kn = 1e-5: dt (CFL) is ~100 tau, the relaxation factor
    # 1 - dt/tau amplifies the non-equilibrium moments within a few steps
    Ue, te, _ = run(1e-5, orc.SRC_EXPLICIT, 40)
    Qe = orc.cons2prim_field(Ue).reshape(-1, system)
    assert not np.all(np.isfinite(Ue)) or np.abs(Qe[:, -1]).max() > 1e3
    # implicit: realizable to t_end and close to the Euler solution
    Ui, ti, hi = run(1e-5, orc.SRC_POINT_IMPLICIT)
    assert ti == pytest.approx(tend)
    Qi = orc.cons2prim_field(Ui).reshape(-1, system)
    assert np.all(np.isfinite(Qi)) and Qi[:, 0].min() > 0
    err_i = np.abs(Qi[:, 0] - ex[:, 0]).mean()
    U3, t3, _ = run(1e-3, orc.SRC_EXPLICIT)
    err_3 = np.abs(orc.cons2prim_field(U3).reshape(-1, system)[:, 0] - ex[:, 0]).mean()
    print(system, "L1(rho - Euler): implicit Kn=1e-5", err_i, "explicit Kn=1e-3", err_3)
    assert err_i < err_3
