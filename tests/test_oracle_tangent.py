"""Pins of the oracle's forward-mode tangent (the same oracle source compiled
with dual numbers), which checks the CUDA adjoint:

  * its primal is bitwise the plain oracle's trajectory;
  * its tangent matches central finite differences of the plain oracle in
    every kind of direction the adjoint differentiates: the state, an
    imposed inflow state (the jets' Mach number), and tau_ref;
  * it is linear in the direction (J(a v + b w) = a Jv + b Jw);
  * a uniform Maxwellian at rest under periodic BCs has zero tangent with
    respect to tau_ref (the BGK source vanishes there)."""
import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import jets_oracle_cfg

pytestmark = pytest.mark.filterwarnings("ignore")


def jets_case(orc, n=14, planar=True, seed=0):
    setup = wl.jets_setup(Kn=0.1)
    prim = wl.jets_like_field(n, n, setup, rng=np.random.default_rng(seed),
                              uz_beam=0.0 if planar else 0.7)
    U = orc.prim2cons_field(prim)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = []
    X = U
    for _ in range(3):
        dts.append(orc.dt(cfg, X, 0.0, 10.0))
        X = orc.step(cfg, X, dts[-1])
    return setup, cfg, U, np.array(dts)


def run_plain(orc, cfg, U, dts):
    for dt in dts:
        U = orc.step(cfg, U, dt)
    return U


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_tangent_primal_is_the_oracle(orc):
    setup, cfg, U, dts = jets_case(orc)
    ref = run_plain(orc, cfg, U, dts)
    out, _ = orc.tangent_run(orc.tangent_cfg(cfg), U, np.zeros_like(U), dts)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("planar", [True, False])
def test_tangent_state_direction_vs_fd(orc, planar):
    """A smooth state (every difference resolved, so that finite differences
    stay on the branch of every limiter and clamp) in the jets' boundary
    set-up; a random relative perturbation of every conserved moment."""
    n = 14
    setup = wl.jets_setup(Kn=0.1)
    prim = wl.smooth_field14(np.random.default_rng(4), n, n, planar=planar)
    U = orc.prim2cons_field(prim)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = [orc.dt(cfg, U, 0.0, 10.0)] * 3
    rng = np.random.default_rng(1)
    V = U * rng.standard_normal(U.shape) * 1e-2
    _, tan = orc.tangent_run(orc.tangent_cfg(cfg), U, V, dts)
    h = 1e-6
    fd = (run_plain(orc, cfg, U + h * V, dts) - run_plain(orc, cfg, U - h * V, dts)) / (2 * h)
    assert rel(tan, fd) < 1e-6, rel(tan, fd)


def test_tangent_inflow_state_vs_fd(orc):
    """d/dM of the left jet's Mach number: the imposed state's u_x moves by
    sqrt(5 T / 3) per unit Mach."""
    setup, cfg, U, dts = jets_case(orc)
    d = np.zeros((4, 1 + orc.MAX_SPANS, 14))
    d[0, 1, 1] = np.sqrt(5.0 / 3.0)
    _, tan = orc.tangent_run(orc.tangent_cfg(cfg, d_states=d), U, np.zeros_like(U), dts)
    h = 1e-6

    def moved(sign):
        s2 = wl.jets_setup(mach=(3.0 + sign * h, 3.0), Kn=0.1)
        return run_plain(orc, jets_oracle_cfg(orc, 14, 14, s2), U, dts)

    fd = (moved(+1) - moved(-1)) / (2 * h)
    assert np.linalg.norm(fd) > 0
    assert rel(tan, fd) < 1e-6, rel(tan, fd)


def test_tangent_tau_ref_vs_fd(orc):
    setup, cfg, U, dts = jets_case(orc)
    _, tan = orc.tangent_run(orc.tangent_cfg(cfg, d_tau_ref=1.0), U, np.zeros_like(U), dts)
    h = 1e-7 * setup["tau_ref"]

    def moved(sign):
        c2 = jets_oracle_cfg(orc, 14, 14, setup)
        c2.tau_ref = setup["tau_ref"] + sign * h
        return run_plain(orc, c2, U, dts)

    fd = (moved(+1) - moved(-1)) / (2 * h)
    assert np.linalg.norm(fd) > 0
    assert rel(tan, fd) < 1e-6, rel(tan, fd)


def test_tangent_is_linear(orc):
    setup, cfg, U, dts = jets_case(orc, n=10)
    rng = np.random.default_rng(2)
    v, w = U * rng.standard_normal((2,) + U.shape) * 1e-3
    tc = orc.tangent_cfg(cfg)
    _, jv = orc.tangent_run(tc, U, v, dts)
    _, jw = orc.tangent_run(tc, U, w, dts)
    _, jvw = orc.tangent_run(tc, U, 2.0 * v - 3.0 * w, dts)
    assert rel(jvw, 2.0 * jv - 3.0 * jw) < 1e-12


def test_tangent_uniform_maxwellian_tau(orc):
    n = 8
    sides = [{"type": orc.BC_PERIODIC}] * 4
    cfg = orc.make_cfg(system=14, nx=n, ny=n, tau_model=orc.TAU_HARDSPHERE, tau_ref=0.3,
                       sides=sides)
    U = orc.prim2cons_field(np.broadcast_to(wl.maxwellian14(1.0, 0.0, 0.0, 1.0), (n, n, 14)))
    _, tan = orc.tangent_run(orc.tangent_cfg(cfg, d_tau_ref=1.0), U, np.zeros_like(U),
                             [1e-3, 1e-3])
    assert np.abs(tan).max() == 0.0


def test_tangent_sod_1d_vs_fd(orc):
    n = 64
    prim = wl.sod_prim(14, n)[None]
    U = orc.prim2cons_field(prim)
    cfg = orc.make_cfg(system=14, nx=n, ny=1, tau_model=2, tau_ref=wl.sod_tau_ref(0.05))
    X, dts = U, []
    for _ in range(6):
        dts.append(orc.dt(cfg, X, 0.0, 1.0))
        X = orc.step(cfg, X, dts[-1])
    _, tan = orc.tangent_run(orc.tangent_cfg(cfg, d_tau_ref=1.0), U, np.zeros_like(U), dts)
    h = 1e-7 * cfg.tau_ref

    def moved(sign):
        c2 = orc.make_cfg(system=14, nx=n, ny=1, tau_model=2,
                          tau_ref=wl.sod_tau_ref(0.05) + sign * h)
        return run_plain(orc, c2, U, dts)

    fd = (moved(+1) - moved(-1)) / (2 * h)
    assert rel(tan, fd) < 1e-6, rel(tan, fd)


# ------------------------------------------------------------------ frozen limiter
def test_frozen_limiter_tangent_primal_and_first_order(orc):
    """The frozen-limiter linearisation (phi held constant in the derivative)
    leaves the primal bitwise unchanged, equals the exact tangent with
    first-order reconstruction (no limiter), and is linear."""
    setup, cfg, U, dts = jets_case(orc)
    ref = run_plain(orc, cfg, U, dts)
    rng = np.random.default_rng(8)
    v, w = U * rng.standard_normal((2,) + U.shape) * 1e-3
    out, jv = orc.tangent_run(orc.tangent_cfg(cfg, frozen_limiter=True), U, v, dts)
    assert np.array_equal(out, ref)
    _, jw = orc.tangent_run(orc.tangent_cfg(cfg, frozen_limiter=True), U, w, dts)
    _, jvw = orc.tangent_run(orc.tangent_cfg(cfg, frozen_limiter=True), U, 2 * v - 3 * w, dts)
    assert rel(jvw, 2 * jv - 3 * jw) < 1e-12
    c1 = orc.make_cfg(system=14, nx=14, ny=14, order=1, tau_model=2, tau_ref=setup["tau_ref"],
                      rho_ref=setup["rho_ref"], T_ref=setup["T_ref"],
                      sides=[{"type": 0, "spans": [(*setup["slot"], setup["left"])]}, {"type": 0},
                             {"type": 0, "spans": [(*setup["slot"], setup["bottom"])]},
                             {"type": 0}])
    _, a = orc.tangent_run(orc.tangent_cfg(c1), U, v, dts)
    _, b = orc.tangent_run(orc.tangent_cfg(c1, frozen_limiter=True), U, v, dts)
    assert np.array_equal(a, b)


def test_frozen_limiter_tangent_saturated_limiter_vs_fd(orc):
    """Where every field alternates from cell to cell, every shared limiter is
    0 on a neighbourhood of the state (dm dp < 0), so holding phi constant
    changes nothing: the frozen tangent equals the exact tangent and central
    differences of the MUSCL step (periodic 1D 14-moment tube)."""
    n = 24
    q = wl.maxwellian14(1.0, 0.1, 0.0, 1.0)
    prim = np.broadcast_to(q, (1, n, 14)).copy()
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    rng = np.random.default_rng(3)
    amp = 0.05 * (1 + 0.3 * rng.random(n))
    prim[0, :, 0] *= 1 + amp * sgn
    prim[0, :, 1] += 0.02 * amp * sgn
    prim[0, :, 4] *= 1 + 0.5 * amp * sgn
    prim[0, :, 7] *= 1 - 0.4 * amp * sgn
    prim[0, :, 9] *= 1 + 0.3 * amp * sgn
    prim[0, :, 10] += 0.01 * amp * sgn
    prim[0, :, 13] *= 1 + 0.8 * amp * sgn
    U = orc.prim2cons_field(prim)
    cfg = orc.make_cfg(system=14, nx=n, ny=1, order=2, tau_model=1, tau_ref=0.2,
                       sides=[{"type": 1}] * 4)
    dts = [orc.dt(cfg, U, 0.0, 10.0)]
    V = U * rng.standard_normal(U.shape) * 1e-3
    _, exact = orc.tangent_run(orc.tangent_cfg(cfg), U, V, dts)
    _, frozen = orc.tangent_run(orc.tangent_cfg(cfg, frozen_limiter=True), U, V, dts)
    assert np.array_equal(exact, frozen)
    h = 1e-6
    fd = (run_plain(orc, cfg, U + h * V, dts) - run_plain(orc, cfg, U - h * V, dts)) / (2 * h)
    assert rel(frozen, fd) < 1e-6, rel(frozen, fd)
