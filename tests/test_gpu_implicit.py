"""Point-implicit BGK source (backward-Euler relaxation after each explicit
stage) on the GPU against the FP64 oracle with the same source scheme:

  * FP64 1D tubes, 5- and 14-moment Sod at Kn = 1e-5 (dt ~ 100 tau at the
    CFL step), per-step parity along the oracle's trajectory, and a free run
    to t = 0.2 that stays realizable;
  * FP64 2D crossed jets at Kn = 1e-5, planar and general states, one step
    and a short per-step trajectory;
  * mixed precision (2D and batched tubes), one step from the oracle's state;
  * the setter's errors, and the adjoint refusing the implicit source.

Errors are normwise per field, measured against the larger of the field's
norm and its tensor family's RMS (a non-equilibrium component that the
relaxation drives to ~g = 1/(1 + dt/tau) of its size, e.g. P_xy in a beam
along x, is measured against the pressure tensor's size: the relaxed value
is a difference of equilibrium-sized numbers).  Bars: FP64 max(1e-12, 10x
the oracle step's change under a 1e-16 data perturbation), forward Euler
1e-12 outright; mixed max(1e-4, 10x the change under a 1e-7 perturbation)
at Kn = 1e-3 (dt ~ 16 tau in the jets: the explicit source is unstable
there).  Closer to equilibrium (Kn = 1e-5) the mixed path's per-step error
grows to ~1e-4 and the floor is 1e-3, measured and unchanged by sending every
face state to FP64: the relaxed non-equilibrium moments are then tiny, their
FP32 increments carry noise at the size of the conserved increment, and the
shared most-stringent limiter takes its minimum over those noise-level
ratios, so the reconstruction slope of every field follows FP32 noise."""
import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import (aos_to_soa, cons_field, field_rel_err, jets_gpu_solver, jets_oracle_cfg,
                         soa_to_aos)
from tests.test_gpu_parity import free_run_drift, gpu_cons, per_step_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12
KN = 1e-5


@pytest.fixture(scope="module")
def mx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as m
    m.lib()
    return m


FAMILIES14 = [[0], [1, 2, 3], [4, 5, 6, 7, 8, 9], [10, 11, 12], [13]]


def fam_err(got, ref):
    """(..., nf) arrays -> per-field normwise error, denominators floored by
    the RMS of the field's tensor family (5-moment: each field its own)."""
    nf = ref.shape[-1]
    a, b = got.reshape(-1, nf), ref.reshape(-1, nf)
    rms = np.sqrt((b * b).mean(axis=0))
    fl = rms.copy()
    if nf == 14:
        for f in FAMILIES14:
            fl[f] = rms[f].max()
    den = np.maximum(np.linalg.norm(b, axis=0), fl * np.sqrt(b.shape[0]))
    num = np.linalg.norm(a - b, axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))


def sensitivity(orc, cfg, U, dt, rng, eps):
    """Per-field change (fam_err) of one oracle step when every primitive of
    the input is perturbed by eps relative."""
    prim = orc.cons2prim_field(U)
    Up = orc.prim2cons_field(prim * (1 + eps * rng.choice([-1.0, 1.0], size=prim.shape)))
    return fam_err(orc.step(cfg, Up, dt), orc.step(cfg, U, dt))


def per_step(mx, s, orc, cfg, U, nsteps, t_end, rng, floor, eps):
    """Every step of the GPU path from the oracle's state (same dt) against
    the oracle's next state: fam_err <= max(floor, 10x sensitivity(eps))."""
    worst, t = 0.0, 0.0
    for k in range(nsteps):
        dt = orc.dt(cfg, U, t, t_end)
        U1 = orc.step(cfg, U, dt)
        sens = sensitivity(orc, cfg, U, dt, rng, eps)
        s.set_state(aos_to_soa(U), kind="conserved")
        s.step_dt([dt])
        e = fam_err(gpu_cons(s), U1)
        assert (e <= np.maximum(floor, 10 * sens)).all(), (k, e, sens)
        worst = max(worst, e.max())
        U, t = U1, t + dt
    return worst


def sod_pair(mx, orc, system, nx, order, integ, precision="fp64"):
    prim = wl.sod_prim(system, nx)
    s = mx.Solver(system=system, nx=nx, ny=1, order=order, integrator=integ,
                  precision=precision)
    s.set_state(aos_to_soa(prim[None]))
    s.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(KN), 1.0, 1.0)
    s.set_source_scheme("point_implicit")
    cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=order,
                       integrator=0 if integ == "fe" else 1, tau_model=2,
                       tau_ref=wl.sod_tau_ref(KN), source_scheme=orc.SRC_POINT_IMPLICIT)
    return s, cfg, cons_field(orc, prim[None])


@pytest.mark.parametrize("system,order,integ", [(5, 1, "fe"), (5, 2, "rk2"), (14, 2, "rk2"),
                                                (14, 1, "fe")])
def test_sod_per_step_parity(mx, orc, system, order, integ):
    s, cfg, U = sod_pair(mx, orc, system, 400, order, integ)
    dt_o = orc.dt(cfg, U, 0.0, 0.2)
    tau = wl.sod_tau_ref(KN)
    assert dt_o > 50 * tau            # the regime where an explicit source is unstable
    if integ == "fe":
        worst, U2, t2 = per_step_parity(mx, s, orc, cfg, U, 120, 0.2)
    else:
        worst = per_step(mx, s, orc, cfg, U, 120, 0.2, np.random.default_rng(1), TOL, 1e-16)
    print(f"system {system} order {order} {integ}: per-step worst {worst:.2e}")


@pytest.mark.parametrize("system", [5, 14])
def test_sod_free_run_realizable(mx, orc, system):
    """Both sides march to t = 0.2 on their own clocks; the GPU state stays
    finite and realizable, and its density is close to the oracle's (the
    shared limiter lets free trajectories separate at noise level, so the
    comparison is an L1 bound, not the 1e-12 gate)."""
    nx = 400
    s, cfg, U = sod_pair(mx, orc, system, nx, 2, "rk2")
    t, n = s.step(10 ** 6, 0.2)
    assert t == pytest.approx(0.2, rel=1e-14)
    d = s.diagnostics()
    assert d["n_nonfinite"] == 0 and d["n_nonpositive"] == 0
    Uo, to, hist = orc.run(cfg, U, 0.0, 0.2, 10 ** 6)
    G = gpu_cons(s)
    l1 = np.abs(G[0, :, 0] - Uo[0, :, 0]).sum() / np.abs(Uo[0, :, 0]).sum()
    print(f"system {system}: {n} GPU steps, {len(hist)} oracle steps, L1 density drift {l1:.2e}")
    assert l1 <= 1e-3


def jets_pair(mx, orc, n, m, precision="fp64", uz=0.0, kn=KN):
    setup = wl.jets_setup(Kn=kn)
    prim = wl.jets_like_field(n, m, setup, uz_beam=uz)
    s = jets_gpu_solver(mx, n, m, setup, precision=precision)
    s.set_source_scheme("point_implicit")
    cfg = jets_oracle_cfg(orc, n, m, setup)
    cfg.source_scheme = orc.SRC_POINT_IMPLICIT
    return s, cfg, cons_field(orc, prim)


@pytest.mark.parametrize("nx,ny,uz", [(40, 37, 0.0), (31, 17, 0.0), (33, 30, 0.8)])
def test_jets2d_one_step(mx, orc, nx, ny, uz):
    s, cfg, U = jets_pair(mx, orc, nx, ny, uz=uz)
    s.set_state(aos_to_soa(U), kind="conserved")
    assert s.diagnostics()["planar"] == int(uz == 0.0)
    dt_o = orc.dt(cfg, U, 0.0, 10.0)
    t, n = s.step(1, 10.0)
    assert t == pytest.approx(dt_o, rel=TOL)
    sens = sensitivity(orc, cfg, U, dt_o, np.random.default_rng(2), 1e-16)
    err = fam_err(gpu_cons(s), orc.step(cfg, U, dt_o))
    print(f"jets one step {nx}x{ny} uz={uz}: {err.max():.2e} (sensitivity {sens.max():.2e})")
    assert (err <= np.maximum(TOL, 10 * sens)).all(), (err, sens)


def test_jets2d_trajectory(mx, orc):
    s, cfg, U = jets_pair(mx, orc, 48, 48)
    worst = per_step(mx, s, orc, cfg, U, 20, 10.0, np.random.default_rng(3), TOL, 1e-16)
    print(f"jets Kn=1e-5 implicit: per-step worst {worst:.2e}")


@pytest.mark.parametrize("uz,kn", [(0.0, 1e-3), (0.8, 1e-3), (0.0, 1e-5)])
def test_mixed_2d_per_step(mx, orc, uz, kn):
    n = 48
    s, cfg, U = jets_pair(mx, orc, n, n, precision="mixed", uz=uz, kn=kn)
    worst = per_step(mx, s, orc, cfg, U, 4, 10.0, np.random.default_rng(5),
                     1e-4 if kn >= 1e-4 else 1e-3, 1e-7)
    assert s.diagnostics()["planar"] == int(uz == 0.0)
    print(f"mixed 2D implicit uz={uz} Kn={kn}: per-step error max {worst:.2e}")


def test_mixed_tubes_per_step(mx, orc):
    tubes = [(120, 1e-3, 8.0), (257, 3e-4, 5.0), (64, KN, 12.0)]
    b = mx.Batch([t[0] for t in tubes], [1.0] * len(tubes), system=14, precision="mixed")
    for i, (nc, kn, r) in enumerate(tubes):
        b.set_tube_relaxation(i, mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
    b.set_source_scheme("point_implicit")
    Us = [cons_field(orc, wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None]) for (nc, kn, r) in tubes]
    cfgs = [orc.make_cfg(system=14, nx=nc, ny=1, tau_model=2, tau_ref=wl.sod_tau_ref(kn),
                         source_scheme=orc.SRC_POINT_IMPLICIT) for (nc, kn, r) in tubes]
    rng = np.random.default_rng(8)
    worst = 0.0
    for step in range(8):
        b.set_state(b.pack([aos_to_soa(U)[:, 0] for U in Us]), kind="conserved")
        b.run(1, 0.2)
        out = b.unpack(b.get_moments("conserved"))
        for i in range(len(tubes)):
            dt = orc.dt(cfgs[i], Us[i], 0.0, 0.2)
            sens = sensitivity(orc, cfgs[i], Us[i], dt, rng, 1e-7)
            Us[i] = orc.step(cfgs[i], Us[i], dt)
            err = fam_err(soa_to_aos(out[i][:, None, :]), Us[i])
            floor = 1e-4 if tubes[i][1] >= 1e-4 else 1e-3
            assert (err <= np.maximum(floor, 10 * sens)).all(), (step, i, err, sens)
            worst = max(worst, err.max())
    print(f"mixed tubes implicit: per-step error max {worst:.2e}")


def test_setter_and_adjoint_guard(mx, orc):
    setup = wl.jets_setup(Kn=0.1)
    s = jets_gpu_solver(mx, 16, 16, setup)
    with pytest.raises(mx.MaxentError):
        s.set_source_scheme(2)
    s.set_state(aos_to_soa(wl.jets_like_field(16, 16, setup)))
    s.set_source_scheme("point_implicit")
    with pytest.raises(mx.MaxentError):
        s.adjoint_record([1e-5])
    s.set_source_scheme("explicit")
    s.adjoint_record([1e-5])
