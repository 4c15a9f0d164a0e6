"""Scheme-level pins of the oracle (CPU only): conservation, symmetry, the
homogeneous BGK relaxation, the Euler limit and the consistency of the
block/window machinery used for sampled full-size parity."""
import math

import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl


def cons_field(orc, prim):
    sh = prim.shape
    flat = prim.reshape(-1, sh[-1])
    return np.array([orc.prim2cons(q) for q in flat]).reshape(sh)


def prim_field(orc, U):
    sh = U.shape
    flat = U.reshape(-1, sh[-1])
    return np.array([orc.cons2prim(u) for u in flat]).reshape(sh)


def periodic_sides(ny):
    s = [{"type": 1}, {"type": 1}, {"type": 1}, {"type": 1}]
    return s


def jets_cfg(orc, n, setup, order=2, integ=1):
    lo, hi = setup["slot"]
    sides = [
        {"type": 0, "spans": [(lo, hi, setup["left"])]},
        {"type": 0},
        {"type": 0, "spans": [(lo, hi, setup["bottom"])]},
        {"type": 0},
    ]
    return orc.make_cfg(system=14, nx=n, ny=n, order=order, integrator=integ,
                        tau_model=2, tau_ref=setup["tau_ref"], rho_ref=setup["rho_ref"],
                        T_ref=setup["T_ref"], sides=sides)


# ------------------------------------------------------------------ uniform
@pytest.mark.parametrize("system,ny,per", [(5, 1, 0), (5, 1, 1), (14, 1, 0), (14, 6, 1), (14, 6, 0)])
def test_uniform_state_stays_bitwise_uniform(orc, system, ny, per):
    rng = np.random.default_rng(20)
    Q = (wl.random_prim5 if system == 5 else wl.random_prim14)(rng, 1)[0]
    nx = 8
    U = np.broadcast_to(orc.prim2cons(Q), (ny, nx, Q.size)).copy()
    sides = [{"type": per}] * 4
    cfg = orc.make_cfg(system=system, nx=nx, ny=ny, tau_model=0, sides=sides)
    dt = orc.dt(cfg, U, 0.0, 1.0)
    U2 = orc.step(cfg, U, dt)
    assert np.array_equal(U2, U)


# ------------------------------------------------------------------ conservation
def test_conservation_periodic_2d_with_bgk(orc):
    """Mass, momentum and energy (trace of the second moment) are conserved
    to round-off: C_1 = C_i = 0, tr C_ij = 0 (Sec. 2.4) and the FV
    differences telescope under periodic BCs."""
    rng = np.random.default_rng(21)
    prim = wl.smooth_field14(rng, 16, 12, amp=0.4)
    U = cons_field(orc, prim)
    cfg = orc.make_cfg(system=14, nx=16, ny=12, tau_model=1, tau_ref=0.05,
                       sides=periodic_sides(12))
    tot0 = U.reshape(-1, 14).sum(0)
    t = 0.0
    for _ in range(30):
        dt = orc.dt(cfg, U, t, 10.0)
        U = orc.step(cfg, U, dt)
        t += dt
    tot = U.reshape(-1, 14).sum(0)
    for k in (0, 1, 2, 3):
        assert abs(tot[k] - tot0[k]) <= 1e-13 * np.abs(U[..., 0]).sum()
    e0 = tot0[4] + tot0[7] + tot0[9]
    e = tot[4] + tot[7] + tot[9]
    assert abs(e - e0) <= 1e-13 * abs(e0)
    # the non-conserved moments did relax / evolve
    assert abs(tot[13] - tot0[13]) > 1e-6 * abs(tot0[13])


def test_conservation_periodic_5moment(orc):
    rng = np.random.default_rng(22)
    x = (np.arange(40) + 0.5) / 40
    prim = np.array([wl.maxwellian5(1 + 0.3 * math.sin(2 * math.pi * xi),
                                    0.2 * math.cos(2 * math.pi * xi), 1.0) for xi in x])
    prim[:, 3] += 0.05 * np.sin(4 * math.pi * x)
    U = cons_field(orc, prim[None])
    cfg = orc.make_cfg(system=5, nx=40, ny=1, tau_model=1, tau_ref=0.1,
                       sides=[{"type": 1}] * 4)
    tot0 = U.reshape(-1, 5).sum(0)
    t = 0.0
    for _ in range(50):
        dt = orc.dt(cfg, U, t, 10.0)
        U = orc.step(cfg, U, dt); t += dt
    tot = U.reshape(-1, 5).sum(0)
    np.testing.assert_allclose(tot[:3], tot0[:3], rtol=1e-13, atol=1e-13 * abs(tot0[0]))


# ------------------------------------------------------------------ symmetry
def mirror5(P):
    P = P[:, ::-1].copy()
    P[..., 1] *= -1; P[..., 3] *= -1
    return P


def mirror14(P):
    P = P[:, ::-1].copy()
    for k in (1, 5, 6, 10):
        P[..., k] *= -1
    return P


@pytest.mark.parametrize("system,order,integ,steps", [(5, 1, 0, 120), (14, 2, 1, 60)])
def test_sod_mirror_symmetry(orc, system, order, integ, steps):
    """x -> 1-x with u, q_x (and P_xy, P_xz) reversed maps the Sod solution
    onto the mirrored problem (swapped left/right states)."""
    nx = 64
    prim = wl.sod_prim(system, nx)[None]
    mir = mirror5 if system == 5 else mirror14
    U = cons_field(orc, prim)
    Um = cons_field(orc, mir(prim))
    cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=order, integrator=integ,
                       tau_model=2, tau_ref=wl.sod_tau_ref(0.05))
    t = 0.0
    for _ in range(steps):
        dt = orc.dt(cfg, U, t, 1.0)
        dtm = orc.dt(cfg, Um, t, 1.0)
        assert dt == pytest.approx(dtm, rel=1e-13)
        U = orc.step(cfg, U, dt); Um = orc.step(cfg, Um, dt); t += dt
    Pm = prim_field(orc, Um)
    P = prim_field(orc, U)
    Pmm = mir(Pm)
    scale = np.abs(P).max(axis=(0, 1)) + 1e-300
    assert np.max(np.abs(Pmm - P) / scale) < 1e-11


def test_jets_diagonal_symmetry(orc):
    """The crossed-jets set-up is symmetric about the diagonal x = y: the
    solution satisfies U(x,y) = swap_xy U(y,x)."""
    setup = wl.jets_setup(Kn=0.1)
    n = 20
    cfg = jets_cfg(orc, n, setup)
    U = cons_field(orc, wl.jets_initial(n, n, setup))
    t = 0.0
    for _ in range(12):
        dt = orc.dt(cfg, U, t, 10.0)
        U = orc.step(cfg, U, dt); t += dt
    P = prim_field(orc, U)
    sw = [0, 2, 1, 3, 7, 5, 8, 4, 6, 9, 11, 10, 12, 13]
    PT = P.transpose(1, 0, 2)[..., sw]
    scale = np.abs(P).max(axis=(0, 1)) + 1e-300
    assert np.max(np.abs(PT - P) / scale) < 1e-11
    assert P[..., 0].max() > 10 * setup["background"][0]     # jets entered


# ------------------------------------------------------------------ relaxation
@pytest.mark.parametrize("integ", [0, 1])
def test_homogeneous_bgk_relaxation_discrete_factor(orc, integ):
    """A uniform non-equilibrium state relaxes as U - U_M -> g (U - U_M) per
    step, g = 1 - dt/tau (FE) or 1 - dt/tau + dt^2/(2 tau^2) (midpoint RK2),
    with U_M the Maxwellian at the (invariant) density, velocity and
    temperature (moments by Gauss-Hermite quadrature)."""
    from numpy.polynomial.hermite_e import hermegauss
    rng = np.random.default_rng(23)
    Q = wl.random_prim14(rng, 1)[0]
    tau = 0.3
    cfg = orc.make_cfg(system=14, nx=4, ny=4, tau_model=1, tau_ref=tau, integrator=integ,
                       sides=[{"type": 1}] * 4)
    U = np.broadcast_to(orc.prim2cons(Q), (4, 4, 14)).copy()
    x, wq = hermegauss(6); wq = wq / math.sqrt(2 * math.pi)
    T = (Q[4] + Q[7] + Q[9]) / (3 * Q[0])
    V = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3) * math.sqrt(T) + Q[1:4]
    W = np.einsum("a,b,c->abc", wq, wq, wq).reshape(-1) * Q[0]
    from tests.test_oracle_pins import psi14
    UM = (W[:, None] * psi14(V)).sum(0)
    d0 = U[0, 0] - UM
    dt = 0.07
    n = 10
    for _ in range(n):
        U = orc.step(cfg, U, dt)
    g = 1 - dt / tau + (dt * dt / (2 * tau * tau) if integ == 1 else 0.0)
    np.testing.assert_allclose(U[0, 0] - UM, g ** n * d0, rtol=1e-9, atol=1e-11 * abs(UM).max())


# ------------------------------------------------------------------ Euler limit
def exact_riemann(rhoL, uL, pL, rhoR, uR, pR, gam, xi):
    """Exact Riemann solution of the Euler equations (two-shock/rarefaction
    Newton iteration on the star pressure, textbook form) sampled at x/t."""
    aL, aR = math.sqrt(gam * pL / rhoL), math.sqrt(gam * pR / rhoR)
    g1, g2 = (gam - 1) / (2 * gam), (gam + 1) / (2 * gam)

    def f(p, rho, pk, a):
        if p > pk:
            A = 2 / ((gam + 1) * rho); B = (gam - 1) / (gam + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B)), math.sqrt(A / (B + p)) * (1 - (p - pk) / (2 * (B + p)))
        return 2 * a / (gam - 1) * ((p / pk) ** g1 - 1), (p / pk) ** (-g2) / (rho * a)

    p = 0.5 * (pL + pR)
    for _ in range(100):
        fl, dl = f(p, rhoL, pL, aL); fr, dr = f(p, rhoR, pR, aR)
        pn = max(p - (fl + fr + uR - uL) / (dl + dr), 1e-12)
        if abs(pn - p) < 1e-14 * p:
            p = pn; break
        p = pn
    fl, _ = f(p, rhoL, pL, aL); fr, _ = f(p, rhoR, pR, aR)
    us = 0.5 * (uL + uR) + 0.5 * (fr - fl)
    out = np.zeros((len(xi), 3))
    for n, s in enumerate(xi):
        if s <= us:
            if p > pL:
                rs = rhoL * ((p / pL + (gam - 1) / (gam + 1)) / ((gam - 1) / (gam + 1) * p / pL + 1))
                S = uL - aL * math.sqrt(g2 * p / pL + g1)
                out[n] = (rhoL, uL, pL) if s < S else (rs, us, p)
            else:
                als = aL * (p / pL) ** g1
                if s < uL - aL:
                    out[n] = (rhoL, uL, pL)
                elif s > us - als:
                    out[n] = (rhoL * (p / pL) ** (1 / gam), us, p)
                else:
                    u = 2 / (gam + 1) * (aL + (gam - 1) / 2 * uL + s)
                    a = 2 / (gam + 1) * (aL + (gam - 1) / 2 * (uL - s))
                    rho = rhoL * (a / aL) ** (2 / (gam - 1))
                    out[n] = (rho, u, pL * (a / aL) ** (2 * gam / (gam - 1)))
        else:
            if p > pR:
                rs = rhoR * ((p / pR + (gam - 1) / (gam + 1)) / ((gam - 1) / (gam + 1) * p / pR + 1))
                S = uR + aR * math.sqrt(g2 * p / pR + g1)
                out[n] = (rhoR, uR, pR) if s > S else (rs, us, p)
            else:
                ars = aR * (p / pR) ** g1
                if s > uR + aR:
                    out[n] = (rhoR, uR, pR)
                elif s < us + ars:
                    out[n] = (rhoR * (p / pR) ** (1 / gam), us, p)
                else:
                    u = 2 / (gam + 1) * (-aR + (gam - 1) / 2 * uR + s)
                    a = 2 / (gam + 1) * (aR - (gam - 1) / 2 * (uR - s))
                    rho = rhoR * (a / aR) ** (2 / (gam - 1))
                    out[n] = (rho, u, pR * (a / aR) ** (2 * gam / (gam - 1)))
    return out


def test_exact_riemann_solver_sanity():
    # Toro's test 1 star state for gamma = 1.4: p* = 0.30313, u* = 0.92745
    sol = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, np.array([0.927]))
    assert sol[0, 2] == pytest.approx(0.30313, rel=1e-4)


@pytest.mark.parametrize("system,gam,order,integ", [(5, 3.0, 1, 0), (14, 5.0 / 3.0, 2, 1)])
def test_euler_limit_trend(orc, system, gam, order, integ):
    """As Kn -> 0 the BGK source drives the moment system to the Euler
    equations (gamma = 3 for the 1D1V gas, 5/3 for the 3D3V gas): the L1
    distance of the density to the exact Riemann solution decreases
    monotonically over Kn = 1, 0.1, 0.01, 0.001."""
    nx, tend = 160, 0.15
    x = (np.arange(nx) + 0.5) / nx
    ex = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gam, (x - 0.5) / tend)
    errs = []
    for Kn in (1.0, 0.1, 0.01, 0.001):
        U = cons_field(orc, wl.sod_prim(system, nx)[None])
        cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=order, integrator=integ,
                           tau_model=2, tau_ref=wl.sod_tau_ref(Kn))
        U2, t, h = orc.run(cfg, U, 0.0, tend, 200000)
        assert t == pytest.approx(tend)
        errs.append(np.abs(U2[0, :, 0] - ex[:, 0]).mean())
    print(system, errs)
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 0.8 * errs[0]


# ------------------------------------------------------------------ block machinery
def test_window_steps_reproduce_full_step(orc):
    """Sub-windows stepped on margin-4 blocks give exactly the full-grid step
    (this is what sampled parity at large sizes relies on)."""
    setup = wl.jets_setup(Kn=0.1)
    n = 18
    cfg = jets_cfg(orc, n, setup)
    rng = np.random.default_rng(24)
    prim = wl.smooth_field14(rng, n, n, amp=0.3)
    U = cons_field(orc, prim)
    dt = orc.dt(cfg, U, 0.0, 10.0)
    full = orc.step(cfg, U, dt)
    for (i0, j0, w, h) in [(0, 0, 5, 4), (6, 7, 6, 5), (13, 0, 5, 6), (0, 12, 7, 6), (10, 13, 8, 5)]:
        win = orc.window_step(cfg, U, i0, j0, w, h, dt)
        assert np.array_equal(win, full[j0:j0 + h, i0:i0 + w])


def test_window_steps_periodic_and_1d(orc):
    rng = np.random.default_rng(25)
    prim = wl.smooth_field14(rng, 12, 10, amp=0.3)
    U = cons_field(orc, prim)
    cfg = orc.make_cfg(system=14, nx=12, ny=10, tau_model=1, tau_ref=0.2,
                       sides=[{"type": 1}] * 4)
    dt = orc.dt(cfg, U, 0.0, 10.0)
    full = orc.step(cfg, U, dt)
    win = orc.window_step(cfg, U, 9, 7, 3, 3, dt)
    assert np.array_equal(win, full[7:10, 9:12])
    U1 = cons_field(orc, wl.sod_prim(14, 30)[None])
    cfg1 = orc.make_cfg(system=14, nx=30, ny=1)
    dt1 = orc.dt(cfg1, U1, 0.0, 1.0)
    f1 = orc.step(cfg1, U1, dt1)
    assert np.array_equal(orc.window_step(cfg1, U1, 26, 0, 4, 1, dt1), f1[:, 26:30])
    assert np.array_equal(orc.window_step(cfg1, U1, 11, 0, 9, 1, dt1), f1[:, 11:20])


# ------------------------------------------------------------------ realizability
def test_c1_sod5_stays_realizable(orc):
    """The 5-moment Sod tube (1000 cells, Kn = 0.01, first-order HLL, FE,
    CFL 0.5, t = 0.2): every cell ends with rho > 0, P > 0, sigma <= 1."""
    nx = 1000
    U = cons_field(orc, wl.sod_prim(5, nx)[None])
    cfg = orc.make_cfg(system=5, nx=nx, ny=1, order=1, integrator=0, tau_model=2,
                       tau_ref=wl.sod_tau_ref(0.01))
    U2, t, h = orc.run(cfg, U, 0.0, 0.2, 10 ** 6)
    assert t == pytest.approx(0.2)
    P = prim_field(orc, U2)[0]
    assert (P[:, 0] > 0).all() and (P[:, 2] > 0).all()
    assert max(orc.sigma(q) for q in P) <= 1.0 + 1e-12
