"""Discrete adjoint of the 2D 14-moment scheme (planar, FP64) on the GPU,
checked against the oracle's forward-mode tangent (an independent
linearisation of the same discrete map, the oracle source compiled with dual
numbers) by the identity <ybar, J xdot> = <J^T ybar, xdot>, and against
central finite differences of the GPU forward with the step sizes frozen.

Bounds: dot-product identities to 1e-10 relative for one residual and 1e-8
for several steps (the GPU trajectory equals the oracle's to ~1e-13 and the
linearisations follow the same branches); the probe gradient within 1e-4
relative of central differences (h = 1e-4 on the Mach numbers, 1e-4
relative on tau_ref)."""
import math

import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import aos_to_soa, jets_gpu_solver, jets_oracle_cfg, soa_to_aos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as m
    m.lib()
    return m


Z_ODD = [3, 6, 8, 12]


def case(orc, n, seed, smooth=True):
    setup = wl.jets_setup(Kn=0.1)
    rng = np.random.default_rng(seed)
    if smooth:
        prim = wl.smooth_field14(rng, n, n, planar=True)
    else:
        prim = wl.jets_like_field(n, n, setup, rng=rng)
    U = orc.prim2cons_field(prim)                 # (n, n, 14)
    return setup, U, rng


def directions(rng, U):
    """state direction (relative), inflow-state directions for both slots,
    tau_ref direction"""
    xd = U * rng.standard_normal(U.shape) * 1e-2
    xd[..., Z_ODD] = 0.0
    gd = np.zeros((4, 5, 14))
    for side in (0, 2):
        gd[side, 1, [0, 1, 2, 4, 5, 7, 9, 10, 11, 13]] = rng.standard_normal(10)
    return xd, gd, float(rng.standard_normal())


def test_adjoint_residual_dot_product(mx, orc):
    n = 20
    setup, U, rng = case(orc, n, 1)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    s = jets_gpu_solver(mx, n, n, setup)
    s.set_state(aos_to_soa(U), kind="conserved")
    V = rng.standard_normal(U.shape)
    V[..., Z_ODD] = 0.0
    out, gb, tb = s.adjoint_residual(aos_to_soa(U), aos_to_soa(V))
    xd, gd, td = directions(rng, U)
    for name, (x, g, t) in {"state": (xd, gd * 0, 0.0), "inflow": (xd * 0, gd, 0.0),
                            "tau": (xd * 0, gd * 0, td)}.items():
        _, dL = orc.tangent_residual(orc.tangent_cfg(cfg, d_states=g, d_tau_ref=t), U, x)
        lhs = float((V * dL).sum())
        rhs = float((soa_to_aos(out) * x).sum() + (gb * g).sum() + tb * t)
        scale = abs(lhs) + 1e-300
        print(f"residual <V, L' x> {name}: {lhs:.12e} vs {rhs:.12e}")
        assert abs(lhs - rhs) <= 1e-10 * scale, (name, lhs, rhs)


@pytest.mark.parametrize("smooth", [True, False])
def test_adjoint_steps_dot_product(mx, orc, smooth):
    """Several RK2 steps, reverse sweep vs the oracle's tangent."""
    n = 20
    setup, U, rng = case(orc, n, 2, smooth)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = []
    X = U
    for _ in range(5):
        dts.append(orc.dt(cfg, X, 0.0, 10.0))
        X = orc.step(cfg, X, dts[-1])
    s = jets_gpu_solver(mx, n, n, setup)
    s.set_state(aos_to_soa(U), kind="conserved")
    s.adjoint_record(dts)
    Ug = soa_to_aos(s.get_moments("conserved"))
    assert np.abs(Ug - X).max() <= 1e-11 * np.abs(X).max()
    ybar = rng.standard_normal(U.shape)
    ybar[..., Z_ODD] = 0.0
    xbar = aos_to_soa(ybar.copy())
    gb, tb = s.adjoint_run(xbar)
    xd, gd, td = directions(rng, U)
    for name, (x, g, t) in {"state": (xd, gd * 0, 0.0), "inflow": (xd * 0, gd, 0.0),
                            "tau": (xd * 0, gd * 0, td)}.items():
        _, jx = orc.tangent_run(orc.tangent_cfg(cfg, d_states=g, d_tau_ref=t), U, x, dts)
        lhs = float((ybar * jx).sum())
        rhs = float((soa_to_aos(xbar) * x).sum() + (gb * g).sum() + tb * t)
        print(f"{'smooth' if smooth else 'jets'} 5 steps <ybar, J x> {name}: {lhs:.12e} vs {rhs:.12e}")
        assert abs(lhs - rhs) <= 1e-8 * (abs(lhs) + 1e-300), (name, lhs, rhs)


@pytest.mark.parametrize("tape", ["keep", "recompute"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("initial", ["rest", "smooth"])
def test_adjoint_probe_gradient_vs_fd(mx, initial, precision, tape):
    """Crossed jets (64^2, 200 RK2 steps, checkpoints every 40): gradient of
    the probe-mean density w.r.t. both Mach numbers and tau_ref against
    central differences of the frozen-dt map.  First-order reconstruction:
    with MUSCL and the shared most-stringent limiter the discrete map is not
    differentiable at the scale of any finite difference (the limiter ratio
    of fields whose differences are near round-off makes finite differences
    diverge as h -> 0); there the adjoint is checked against the oracle's
    tangent instead (test_adjoint_steps_dot_product).  precision "mixed":
    the face states reversed in FP32 from the FP64 tape.  tape "keep": the
    forward march records the whole tape; "recompute": checkpoints every 40
    steps, each segment replayed before its sweep (the two give the same
    gradient up to the order of the segment sums)."""
    from paper_2401_15233_gb300 import adjoint as ad
    prob = ad.JetsProblem(n=64, nsteps=200, ckpt=40, probe=8, initial=initial, order=1,
                          adjoint_precision=precision, tape=tape)
    p0 = prob.params0()
    J, ckpts, dts, s = ad.forward_checkpointed(prob, p0)
    assert prob.tape_kept == (tape == "keep") and len(ckpts) == (0 if tape == "keep" else 5)
    g, _ = ad.backward_checkpointed(prob, s, ckpts, dts)
    assert abs(ad.run_fixed(prob, p0, dts) - J) <= 1e-14 * abs(J)
    hs = [1e-4, 1e-4, 1e-4 * p0[2]]
    fd = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = hs[k]
        fd.append((ad.run_fixed(prob, p0 + e, dts) - ad.run_fixed(prob, p0 - e, dts)) / (2 * hs[k]))
    fd = np.array(fd)
    print(f"{initial} {precision}: probe J {J:.10e} adjoint {g} fd {fd}")
    assert np.all(np.abs(fd) > 0)
    assert np.all(np.abs(g - fd) <= 1e-4 * np.abs(fd)), (g, fd)


def test_adjoint_autograd_function(mx):
    import torch
    from paper_2401_15233_gb300 import adjoint as ad
    prob = ad.JetsProblem(n=48, nsteps=120, ckpt=30, probe=8, initial="rest", order=1)
    p = torch.tensor(prob.params0(), dtype=torch.float64, requires_grad=True)
    J = ad.jets_probe(p, prob)
    J.backward()
    Jd, ckpts, dts, s = ad.forward_checkpointed(prob, prob.params0())
    g, _ = ad.backward_checkpointed(prob, s, ckpts, dts)
    assert float(J) == Jd
    assert np.allclose(p.grad.numpy(), g, rtol=1e-12, atol=0)


def test_adjoint_mixed_matches_fp64(mx, orc):
    """FP32 face-state reverse against the FP64 one, five MUSCL steps: same
    adjoint up to FP32 rounding.  The state has no exact ties between the
    fields' limiter ratios (smooth_field14 makes P_yy = P_zz; P_zz is
    modulated here): at a tie the shared limiter's min has several
    sub-gradients and FP32 and FP64 may pick different ones."""
    n = 20
    setup = wl.jets_setup(Kn=0.1)
    rng = np.random.default_rng(2)
    prim = wl.smooth_field14(rng, n, n, planar=True)
    x = (np.arange(n) + 0.5) / n
    prim[..., 9] *= 1.0 + 0.05 * np.cos(2 * np.pi * x)[None, :]
    U = orc.prim2cons_field(prim)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = []
    X = U
    for _ in range(5):
        dts.append(orc.dt(cfg, X, 0.0, 10.0))
        X = orc.step(cfg, X, dts[-1])
    ybar = rng.standard_normal(U.shape)
    ybar[..., Z_ODD] = 0.0
    res = {}
    for prec in ("fp64", "mixed"):
        s = jets_gpu_solver(mx, n, n, setup)
        s.set_adjoint_precision(prec)
        s.set_state(aos_to_soa(U), kind="conserved")
        s.adjoint_record(dts)
        xbar = aos_to_soa(ybar.copy())
        gb, tb = s.adjoint_run(xbar)
        res[prec] = (xbar, gb, tb)
    a, b = res["fp64"], res["mixed"]
    e = np.linalg.norm(a[0] - b[0]) / np.linalg.norm(a[0])
    eg = np.linalg.norm(a[1] - b[1]) / np.linalg.norm(a[1])
    et = abs(a[2] - b[2]) / abs(a[2])
    print(f"mixed vs fp64 adjoint: state {e:.2e} inflow {eg:.2e} tau {et:.2e}")
    assert e < 1e-4 and eg < 1e-4 and et < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("smooth", [True, False])
def test_adjoint_frozen_limiter_dot_product(mx, orc, smooth, precision):
    """The frozen-limiter adjoint (phi held constant in the derivative), FP64
    and FP32 face-state reverse, five MUSCL RK2 steps, against the oracle's
    tangent with the same linearisation; and it differs from the exact
    adjoint on the non-smooth state (the limiter's derivative matters)."""
    n = 20
    setup, U, rng = case(orc, n, 2, smooth)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = []
    X = U
    for _ in range(5):
        dts.append(orc.dt(cfg, X, 0.0, 10.0))
        X = orc.step(cfg, X, dts[-1])
    s = jets_gpu_solver(mx, n, n, setup)
    s.set_state(aos_to_soa(U), kind="conserved")
    s.set_adjoint_precision(precision)
    s.set_adjoint_limiter(True)
    s.adjoint_record(dts)
    ybar = rng.standard_normal(U.shape)
    ybar[..., Z_ODD] = 0.0
    xbar = aos_to_soa(ybar.copy())
    gb, tb = s.adjoint_run(xbar)
    xd, gd, td = directions(rng, U)
    tol = 1e-8 if precision == "fp64" else 1e-4
    for name, (x, g, t) in {"state": (xd, gd * 0, 0.0), "inflow": (xd * 0, gd, 0.0),
                            "tau": (xd * 0, gd * 0, td)}.items():
        tc = orc.tangent_cfg(cfg, d_states=g, d_tau_ref=t, frozen_limiter=True)
        _, jx = orc.tangent_run(tc, U, x, dts)
        lhs = float((ybar * jx).sum())
        rhs = float((soa_to_aos(xbar) * x).sum() + (gb * g).sum() + tb * t)
        print(f"frozen {precision} {'smooth' if smooth else 'jets'} {name}: {lhs:.12e} vs {rhs:.12e}")
        assert abs(lhs - rhs) <= tol * (abs(lhs) + 1e-300), (name, lhs, rhs)
    if not smooth and precision == "fp64":
        s.set_adjoint_limiter(False)
        xe = aos_to_soa(ybar.copy())
        s.adjoint_run(xe)
        assert not np.allclose(xe, xbar, rtol=1e-6, atol=0)


def test_adjoint_c5_size_slot_probe_vs_fd(mx):
    """The adjoint configuration's size (512^2, 500 RK2 steps, checkpoints
    every 50, Kn = 0.1, from rest) with the probe on the left inflow slot,
    which the left jet crosses from the first steps (the configured probe at
    the centre lies outside the inflows' domain of dependence for 500 steps:
    signals travel ~0.1 of the domain, and adjoint and differences are both
    exactly zero there).  First-order reconstruction (a smooth map, see
    test_adjoint_probe_gradient_vs_fd): against central differences
    (h = 1e-4, frozen dt) on the non-zero components, the FP64 reverse
    within 1e-4 (measured 1.4e-5) and the FP32 face-state reverse within
    1e-3 (measured 2.5e-4 on tau_ref: its FP32 face-state derivatives over
    500 steps); the bottom jet's Mach number cannot reach the probe and its
    derivative is zero in both."""
    from paper_2401_15233_gb300 import adjoint as ad
    prob = ad.JetsProblem(n=512, nsteps=500, ckpt=50, probe=32, initial="rest", order=1,
                          probe_at="left_slot", tape="recompute")
    p0 = prob.params0()
    grads = {}
    for prec in ("fp64", "mixed"):
        prob.adjoint_precision = prec
        J, ckpts, dts, s = ad.forward_checkpointed(prob, p0)
        grads[prec], _ = ad.backward_checkpointed(prob, s, ckpts, dts)
        del s, ckpts
    hs = [1e-4, 1e-4, 1e-4 * p0[2]]
    fd = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = hs[k]
        fd.append((ad.run_fixed(prob, p0 + e, dts) - ad.run_fixed(prob, p0 - e, dts)) / (2 * hs[k]))
    fd = np.array(fd)
    print(f"512^2 slot probe, first order: J {J:.10e}, fd {fd}, fp64 {grads['fp64']}, "
          f"fp32 {grads['mixed']}")
    nz = np.abs(fd) > 0
    assert nz[0] and nz[2] and fd[1] == 0.0
    for prec, g in grads.items():
        tol = 1e-4 if prec == "fp64" else 1e-3
        assert np.all(np.abs(g[nz] - fd[nz]) <= tol * np.abs(fd[nz])), (prec, g, fd)
        assert np.all(np.abs(g[~nz]) <= 1e-12 * np.abs(fd).max()), (prec, g)


def test_adjoint_muscl_dot_product_jets_in_probe(mx, orc):
    """MUSCL (the configured scheme), the developed crossed-jets state with
    the jets through the probe region, 64^2, 12 RK2 steps: the reverse sweep
    against the oracle's independent forward-mode tangent, in a state, an
    inflow-state and a tau_ref direction (<ybar, J x> = <J^T ybar, x>, 1e-8).
    MUSCL's shared most-stringent limiter makes the map non-differentiable at
    the scale of finite differences (they do not converge as h -> 0), so for
    MUSCL this identity, not a difference quotient, is the check."""
    n, nsteps = 64, 12
    setup, U, rng = case(orc, n, 7, smooth=False)
    cfg = jets_oracle_cfg(orc, n, n, setup)
    dts = []
    X = U
    for _ in range(nsteps):
        dts.append(orc.dt(cfg, X, 0.0, 10.0))
        X = orc.step(cfg, X, dts[-1])
    s = jets_gpu_solver(mx, n, n, setup)
    s.set_state(aos_to_soa(U), kind="conserved")
    s.adjoint_record(dts)
    ybar = np.zeros(U.shape)
    lo = (n - 16) // 2
    ybar[lo:lo + 16, lo:lo + 16, 0] = 1.0 / 256.0      # the probe-mean density
    xbar = aos_to_soa(ybar.copy())
    gb, tb = s.adjoint_run(xbar)
    xd, gd, td = directions(rng, U)
    for name, (x, g, t) in {"state": (xd, gd * 0, 0.0), "inflow": (xd * 0, gd, 0.0),
                            "tau": (xd * 0, gd * 0, td)}.items():
        _, jx = orc.tangent_run(orc.tangent_cfg(cfg, d_states=g, d_tau_ref=t), U, x, dts)
        lhs = float((ybar * jx).sum())
        rhs = float((soa_to_aos(xbar) * x).sum() + (gb * g).sum() + tb * t)
        print(f"MUSCL jets 64^2 {nsteps} steps <ybar, J x> {name}: {lhs:.12e} vs {rhs:.12e}")
        assert lhs != 0.0
        assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (name, lhs, rhs)
