"""Gradients of crossed-jets probe outputs by the discrete adjoint, behind a
``torch.autograd.Function`` with checkpointed recomputation.

The map is the FP64 scheme (Sec. 3) marched for ``nsteps`` RK2 steps; the
step sizes are fixed by the CFL condition of the unperturbed forward run and
then held constant, so the gradient is that of the fixed-dt discrete map
(the finite-difference check replays the same step sizes).

Forward: march on the device, recording every dt and keeping the conserved
state every ``ckpt`` steps (device tensors).  Backward: for each segment,
last first, restore its checkpoint, replay it with ``mxe_adjoint_record``
(which keeps U^n and U* of each step on the device) and sweep it in reverse
with ``mxe_adjoint_run``; the adjoint state is carried from segment to
segment on the device.  When the whole tape fits in device memory (GB300:
288 GB; 2 x 500 states of 29 MB for the 512^2 configuration) the forward
march records it directly and the backward sweeps it without replaying.  The C library returns the adjoints of the imposed
inflow primitive states and of tau_ref; the inflow velocity of a jet is
M sqrt(gamma T_jet) along its slot normal, which maps the first onto the
Mach numbers.

PyTorch holds the checkpoints and the adjoint state and averages the probe;
every step of the path runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import (BC_DIRICHLET, ENONFINITE, GHOST_SLOTS, TAU_HARDSPHERE, XLO, YLO,
                MaxentError, Solver)
from . import workloads as wl

GAMMA = 5.0 / 3.0


class JetsProblem:
    """Crossed jets on [0,1]^2, n x n cells; probe = mean density over a
    block of probe x probe cells: centred on (0.5, 0.5), where the jets
    cross (probe_at="centre"), or against the left wall centred on the left
    inflow slot (probe_at="left_slot"), which the left jet reaches from the
    first steps.  Parameters p = (Mach of the left jet, Mach of the bottom
    jet, tau_ref).  initial: "developed" (the synthetic developed
    crossed-jets state of the throughput benchmark, both beams already
    across the domain), "rest" (background at rest, the start of a
    simulation) or "smooth" (a smooth, resolved non-equilibrium gas into
    which the jets blow)."""

    def __init__(self, n=512, Kn=0.1, nsteps=500, ckpt=50, probe=32, mach=(3.0, 3.0),
                 initial="developed", order=2, relax=True, adjoint_precision="fp64",
                 adjoint_limiter="exact", probe_at="centre", tape="auto"):
        if nsteps % ckpt:
            raise ValueError("nsteps must be a multiple of ckpt")
        if initial not in ("developed", "rest", "smooth"):
            raise ValueError("initial must be 'developed', 'rest' or 'smooth'")
        if tape not in ("auto", "keep", "recompute"):
            raise ValueError("tape must be 'auto', 'keep' or 'recompute'")
        # "keep": the forward run records the whole tape (U^n, U* of every
        # step) in device memory and the backward sweeps it directly;
        # "recompute": checkpoints every ckpt steps, each segment replayed
        # before its sweep; "auto": keep when the tape fits in half of the
        # free device memory
        self.tape = tape
        self.initial_kind = initial
        self.order, self.relax = order, relax
        self.adjoint_precision = adjoint_precision
        if adjoint_limiter not in ("exact", "frozen"):
            raise ValueError("adjoint_limiter must be 'exact' or 'frozen'")
        self.adjoint_limiter = adjoint_limiter
        self.n, self.nsteps, self.ckpt = n, nsteps, ckpt
        self.setup = wl.jets_setup(mach=mach, Kn=Kn)
        self.p0 = (float(mach[0]), float(mach[1]), float(self.setup["tau_ref"]))
        lo = (n - probe) // 2
        if probe_at not in ("centre", "left_slot"):
            raise ValueError("probe_at must be 'centre' or 'left_slot'")
        self.probe_at = probe_at
        # probe block: rows (y) [r0, r1), columns (x) [c0, c1)
        self.probe = (lo, lo + probe, lo, lo + probe) if probe_at == "centre" else \
            (lo, lo + probe, 0, probe)
        self.T_jet = self.setup["T_ref"]

    def params0(self):
        return np.array(self.p0)

    def solver(self, p):
        s = Solver(system=14, nx=self.n, ny=self.n, precision="fp64", order=self.order,
                   integrator="rk2", flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4)
        su = wl.jets_setup(mach=(float(p[0]), float(p[1])), Kn=self.setup["Kn"])
        lo, hi = su["slot"]
        s.set_bc(XLO, BC_DIRICHLET, lo, hi, su["left"])
        s.set_bc(YLO, BC_DIRICHLET, lo, hi, su["bottom"])
        if self.relax:
            s.set_relaxation(TAU_HARDSPHERE, float(p[2]), su["rho_ref"], su["T_ref"])
        s.set_adjoint_precision(self.adjoint_precision)
        s.set_adjoint_limiter(self.adjoint_limiter == "frozen")
        return s

    def initial(self):
        """(14, n, n) primitive initial state"""
        if self.initial_kind == "rest":
            prim = wl.jets_initial(self.n, self.n, self.setup)
        elif self.initial_kind == "smooth":
            prim = wl.smooth_field14(np.random.default_rng(0), self.n, self.n, planar=True)
        else:
            prim = wl.jets_like_field(self.n, self.n, self.setup)
        return np.ascontiguousarray(np.moveaxis(prim, -1, 0))

    def probe_of(self, U):
        """mean density over the probe block of a conserved state (14, n, n)"""
        r0, r1, c0, c1 = self.probe
        return U[0, r0:r1, c0:c1].mean()

    def dmach(self):
        """d(imposed u_normal)/dM for each jet"""
        return math.sqrt(GAMMA * self.T_jet)


def run_fixed(prob: JetsProblem, p, dts):
    """J(p) with the step sizes dts held fixed (the finite-difference map)."""
    import torch
    s = prob.solver(p)
    s.set_state(prob.initial())
    s.step_dt(dts)
    U = torch.empty((14, prob.n, prob.n), dtype=torch.float64, device="cuda")
    s.get_moments("conserved", out=U)
    return float(prob.probe_of(U))


def tape_bytes(prob: JetsProblem):
    """device memory of the whole tape: U^n and U* of every step"""
    return 2 * prob.nsteps * 14 * prob.n * (prob.n + 32) * 8


def keeps_tape(prob: JetsProblem):
    if prob.tape != "auto":
        return prob.tape == "keep"
    import torch
    free, _ = torch.cuda.mem_get_info()
    return tape_bytes(prob) <= 0.5 * free


def forward_checkpointed(prob: JetsProblem, p):
    """March nsteps CFL steps from the initial state; returns (J,
    checkpoints, dts, solver).  When the tape is kept (keeps_tape) the
    march records it and there are no checkpoints."""
    import torch
    s = prob.solver(p)
    s.set_state(prob.initial())
    s.set_dt_history(prob.nsteps)
    prob.tape_kept = keeps_tape(prob)
    if prob.tape_kept:
        s.adjoint_record(None, prob.nsteps)
        dts = s.dt_history(prob.nsteps)
        U = torch.empty((14, prob.n, prob.n), dtype=torch.float64, device="cuda")
        s.get_moments("conserved", out=U)
        return float(prob.probe_of(U)), [], dts, s
    # checkpoints every ckpt steps; the last segment is recorded into the
    # one-segment tape as it is marched, so the backward starts on it without
    # a replay
    ckpts = []
    nseg = prob.nsteps // prob.ckpt
    for k in range(nseg):
        U = torch.empty((14, prob.n, prob.n), dtype=torch.float64, device="cuda")
        s.get_moments("conserved", out=U)
        ckpts.append(U)
        if k == nseg - 1:
            s.adjoint_record(None, prob.ckpt)
        else:
            s.step(prob.ckpt, float("inf"), sync=False)
    dts = s.dt_history(prob.nsteps)
    U = torch.empty((14, prob.n, prob.n), dtype=torch.float64, device="cuda")
    s.get_moments("conserved", out=U)
    return float(prob.probe_of(U)), ckpts, dts, s


def backward_checkpointed(prob: JetsProblem, s: Solver, ckpts, dts, gJ=1.0):
    """dJ/dp by the reverse sweep, segment by segment (recomputing each
    segment from its checkpoint, except the last, which the forward left on
    the tape).  With the FP32 face-state reverse, a
    segment whose adjoint leaves the FP32 range (non-finite values) is swept
    again with the FP64 reverse from the same incoming adjoint; the number of
    such segments is left in prob.fp64_fallbacks."""
    import torch
    r0, r1, c0, c1 = prob.probe
    ubar = torch.zeros((14, prob.n, prob.n), dtype=torch.float64, device="cuda")
    ubar[0, r0:r1, c0:c1] = gJ / float((r1 - r0) * (c1 - c0))
    torch.cuda.synchronize()          # written on torch's stream, read on the library's
    G = np.zeros((4, GHOST_SLOTS, 14))
    tb = 0.0
    mixed = prob.adjoint_precision == "mixed"
    prob.fp64_fallbacks = 0
    # the kept tape is one segment of all the steps; otherwise replay each
    # checkpointed segment, last first
    segments = [None] if getattr(prob, "tape_kept", False) else range(len(ckpts) - 1, -1, -1)
    for k in segments:
        if k is not None and k != len(ckpts) - 1:     # the last one is on the tape
            s.set_state(ckpts[k], kind="restore")
            s.adjoint_record(dts[k * prob.ckpt:(k + 1) * prob.ckpt])
        keep = ubar.clone() if mixed else None
        torch.cuda.synchronize()
        try:
            g, t = s.adjoint_run(ubar)
        except MaxentError as e:   # the FP32 reverse left its range: sweep again in FP64
            if not mixed or e.status != ENONFINITE:
                raise
            ubar.copy_(keep)
            torch.cuda.synchronize()
            s.set_adjoint_precision("fp64")
            g, t = s.adjoint_run(ubar)
            s.set_adjoint_precision("mixed")
            prob.fp64_fallbacks += 1
        G += g
        tb += t
    # imposed states: left slot (side XLO, span 0) moves u_x, bottom (YLO) u_y
    dM = prob.dmach()
    return np.array([G[XLO, 1, 1] * dM, G[YLO, 1, 2] * dM, tb]), ubar


def _autograd_function():
    import torch

    class JetsProbeFn(torch.autograd.Function):
        """J = probe-mean density after nsteps, as a function of
        p = (M_left, M_bottom, tau_ref) (a float64 tensor of 3)."""

        @staticmethod
        def forward(ctx, p, prob):
            J, ckpts, dts, s = forward_checkpointed(prob, p.detach().cpu().numpy())
            ctx.prob, ctx.ckpts, ctx.dts, ctx.solver = prob, ckpts, dts, s
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            g, _ = backward_checkpointed(ctx.prob, ctx.solver, ctx.ckpts, ctx.dts, float(gJ))
            ctx.ckpts = None
            return torch.tensor(g, dtype=torch.float64), None

    return JetsProbeFn


_FN = None


def jets_probe(p, prob: JetsProblem):
    """Differentiable probe output: ``jets_probe(p, prob).backward()`` fills
    ``p.grad`` with (dJ/dM_left, dJ/dM_bottom, dJ/dtau_ref)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(p, prob)
