"""Seeded synthetic inputs for the maximum-entropy solver.

Every function here returns *primitive* moment states (or plain parameters)
built from the problem definitions of the paper's test cases; none of the
method's arithmetic (conserved variables, closure, fluxes, wave speeds) lives
in this module.  Both the CUDA path and the CPU oracle consume these inputs.

Primitive layouts
  5-moment : (rho, u, P, q, r)                                   Sec. 2.3
  14-moment: (rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz,
              qx, qy, qz, R)                                     Sec. 2.4
Units are non-dimensional with R_gas = k_B/m = 1, so P = rho T.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA_3D = 5.0 / 3.0     # monatomic gas, a = sqrt(gamma T) (Sec. 6 Mach number)
SOD_SEED = 20240127


def maxwellian5(rho, u, T):
    """1D1V Maxwellian: q = 0, r = 3 P^2/rho (Sec. 2.3)."""
    P = rho * T
    return np.array([rho, u, P, 0.0, 3.0 * P * P / rho])


def maxwellian14(rho, ux, uy, T, uz=0.0):
    """3D3V Maxwellian: P_ij = rho T delta_ij, q = 0, R = 15 P^2/rho (Sec. 2.1)."""
    P = rho * T
    return np.array([rho, ux, uy, uz, P, 0.0, 0.0, P, 0.0, P, 0.0, 0.0, 0.0,
                     15.0 * P * P / rho])


# ---------------------------------------------------------------- Sod tubes
def sod_prim(system: int, nx: int, rhoL=1.0, PL=1.0, rhoR=0.125, PR=0.1,
             x0=0.0, x1=1.0, xd=0.5):
    """Sod shock tube at rest with Maxwellian left/right states (Sec. 4).
    Returns (nx, nf) primitives at cell centres."""
    x = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    out = []
    for xi in x:
        rho, P = (rhoL, PL) if xi < xd else (rhoR, PR)
        T = P / rho
        out.append(maxwellian5(rho, 0.0, T) if system == 5 else maxwellian14(rho, 0.0, 0.0, T))
    return np.array(out)


def sod_tau_ref(Kn: float, T_ref: float = 1.0, L_ref: float = 1.0) -> float:
    """tau at the left state for Kn = lambda_L / D (Sec. 4):
    tau = lambda / v_th with v_th = sqrt(8 T / pi)."""
    return Kn * L_ref / math.sqrt(8.0 * T_ref / math.pi)


def batch_tubes(n_tubes: int = 256, seed: int = SOD_SEED, nmin=512, nmax=8192,
                kn_min=1e-3, kn_max=10.0, ratio_min=4.0, ratio_max=20.0):
    """Batched Sod tubes: per tube (ncells, Kn, density ratio) drawn in that
    order from numpy's default_rng(seed); ncells log-uniform in [nmin, nmax]
    (rounded), Kn log-uniform, ratio uniform.  Right state: rho = P = 1/ratio
    (equal temperature, as in the paper's Sod set-up)."""
    rng = np.random.default_rng(seed)
    tubes = []
    for _ in range(n_tubes):
        nc = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kn = math.exp(rng.uniform(math.log(kn_min), math.log(kn_max)))
        ratio = rng.uniform(ratio_min, ratio_max)
        tubes.append((nc, kn, ratio))
    return tubes


# ---------------------------------------------------------------- crossed jets
def jets_setup(mach=(3.0, 3.0), rho_bg=1e-3, T_bg=1.0, rho_jet=1.0, T_jet=1.0,
               slot=(0.45, 0.55), Kn=0.1, slot_width=0.1):
    """Two crossing supersonic jets (Sec. 6): slots on the left (y in slot,
    velocity +x) and bottom (x in slot, velocity +y) walls, Maxwellian
    inflow at (rho_jet, T_jet, |u| = M sqrt(gamma T)), background at rest.
    Returns a dict with the background primitive, the two inflow
    primitives, slot spans and the relaxation parameters
    (tau_ref = Kn L_ref / sqrt(8 T_ref/pi) with L_ref = slot width,
    rho_ref = rho_jet, T_ref = T_jet)."""
    a = math.sqrt(GAMMA_3D * T_jet)
    left = maxwellian14(rho_jet, mach[0] * a, 0.0, T_jet)
    bottom = maxwellian14(rho_jet, 0.0, mach[1] * a, T_jet)
    bg = maxwellian14(rho_bg, 0.0, 0.0, T_bg)
    return dict(background=bg, left=left, bottom=bottom, slot=slot,
                tau_ref=Kn * slot_width / math.sqrt(8.0 * T_jet / math.pi),
                rho_ref=rho_jet, T_ref=T_jet, Kn=Kn)


def collisionless_jets_setup(n_jets=1, mach=5.0, rho_jet=1.0, T_jet=1.0, bg_ratio=1e-5,
                            jet_width=1.0 / 7.0):
    """Collisionless jets into a near vacuum (Sec. 6): jets of width L/7
    centred on the left wall (and, for two jets, the bottom wall), Mach 5,
    Maxwellian at (rho_jet, T_jet); every other boundary cell holds the
    background, rho_0 = 1e-5 rho_jet at T_jet and rest; no collision source.
    The solution of the homogeneous system is self-similar in the density,
    so rho_jet = 1.  Returns the background and jet primitives and the span."""
    a = math.sqrt(GAMMA_3D * T_jet)
    lo, hi = 0.5 - 0.5 * jet_width, 0.5 + 0.5 * jet_width
    out = dict(background=maxwellian14(bg_ratio * rho_jet, 0.0, 0.0, T_jet),
               left=maxwellian14(rho_jet, mach * a, 0.0, T_jet), slot=(lo, hi),
               n_jets=n_jets)
    if n_jets == 2:
        out["bottom"] = maxwellian14(rho_jet, 0.0, mach * a, T_jet)
    return out


def jets_initial(nx: int, ny: int, setup: dict):
    """Uniform background (ny, nx, 14)."""
    return np.broadcast_to(setup["background"], (ny, nx, 14)).copy()


# ---------------------------------------------------------------- random states
def particle_moments14(w, v):
    """Central moments (rho, u, P, q, R) of a weighted set of particles."""
    rho = w.sum()
    u = (w[:, None] * v).sum(0) / rho
    c = v - u
    c2 = (c * c).sum(1)
    P = np.einsum("p,pi,pj->ij", w, c, c)
    q = (w[:, None] * c * c2[:, None]).sum(0)
    R = (w * c2 * c2).sum()
    return np.array([rho, *u, P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2], *q, R])


def particle_moments5(w, v):
    rho = w.sum()
    u = (w * v).sum() / rho
    c = v - u
    return np.array([rho, u, (w * c ** 2).sum(), (w * c ** 3).sum(), (w * c ** 4).sum()])


def random_prim14(rng, n: int, npart: int = 48, aniso: float = 1.0, drift: float = 1.0,
                  planar: bool = False):
    """n realizable 14-moment states from random particle clouds: two or three
    anisotropic Gaussian beams with random weights.  planar=True zeroes the
    z-odd moments (u_z, P_xz, P_yz, q_z) by mirroring the cloud in z."""
    out = []
    for _ in range(n):
        nb = rng.integers(1, 4)
        ws, vs = [], []
        for b in range(nb):
            m = rng.normal(0, drift, 3)
            L = np.diag(np.exp(rng.normal(0, 0.5 * aniso, 3)))
            Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
            v = rng.normal(size=(npart, 3)) @ (Rm @ L).T + m
            ws.append(rng.uniform(0.2, 1.0, npart) * rng.uniform(0.2, 1.0))
            vs.append(v)
        w = np.concatenate(ws)
        v = np.concatenate(vs)
        if planar:
            w = np.concatenate([w, w])
            v = np.concatenate([v, v * np.array([1, 1, -1])])
        out.append(particle_moments14(w * rng.uniform(0.05, 2.0), v))
    return np.array(out)


def random_prim5(rng, n: int, npart: int = 48):
    out = []
    for _ in range(n):
        nb = rng.integers(1, 4)
        ws, vs = [], []
        for b in range(nb):
            ws.append(rng.uniform(0.2, 1.0, npart) * rng.uniform(0.2, 1.0))
            vs.append(rng.normal(rng.normal(0, 1), math.exp(rng.normal(0, 0.5)), npart))
        out.append(particle_moments5(np.concatenate(ws) * rng.uniform(0.05, 2.0),
                                     np.concatenate(vs)))
    return np.array(out)


def smooth_field14(rng, nx: int, ny: int, amp: float = 0.3, planar: bool = True):
    """A smooth, realizable 2D primitive field: Maxwellian-like background with
    smooth density, velocity and temperature waves plus small non-equilibrium
    parts (heat flux, anisotropy, kurtosis) that keep every cell realizable."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    k = rng.integers(1, 3, size=8)
    ph = rng.uniform(0, 2 * np.pi, size=8)
    f = lambda n: np.sin(2 * np.pi * (k[n] * X + k[(n + 3) % 8] * Y) + ph[n])
    rho = 1.0 + amp * 0.5 * f(0)
    ux = amp * f(1)
    uy = amp * f(2)
    T = 1.0 + amp * 0.4 * f(3)
    P = rho * T
    a = 0.1 * amp * f(4)
    Pxx, Pyy = P * (1 + a), P * (1 - 0.5 * a)
    Pzz = 3 * P - Pxx - Pyy
    Pxy = 0.05 * amp * P * f(5)
    qs = 0.1 * amp
    th = P / rho
    qx = qs * rho * th ** 1.5 * f(6)
    qy = qs * rho * th ** 1.5 * f(7)
    # kurtosis a little above Gaussian so sigma stays well inside (0, 1)
    R = (1.0 + 0.05 * amp * f(0) * f(3)) * 15.0 * P * P / rho
    Z = np.zeros_like(X)
    if planar:
        uz, Pxz, Pyz, qz = Z, Z, Z, Z
    else:     # z-odd moments switched on (small, keeping P positive definite)
        uz = 0.5 * amp * f(5) * f(1)
        Pxz = 0.04 * amp * P * f(2)
        Pyz = 0.03 * amp * P * f(6)
        qz = 0.05 * amp * rho * th ** 1.5 * f(4)
    st = np.stack([rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz, qx, qy, qz, R], axis=-1)
    return st


def maxwellian_mixture14(comps):
    """Central moments of a sum of Maxwellians [(rho_a, (ux, uy, uz), T_a), ...]
    (Gaussian moment identities): P = sum rho_a (T_a I + c c^T),
    q = sum rho_a c (|c|^2 + 5 T_a), R = sum rho_a (|c|^4 + 10 T_a |c|^2 + 15 T_a^2),
    with c = u_a - u the offset of each component from the mixture velocity."""
    rho = sum(c[0] for c in comps)
    u = sum(c[0] * np.asarray(c[1], dtype=float) for c in comps) / rho
    P = np.zeros((3, 3)); q = np.zeros(3); R = 0.0
    for ra, ua, Ta in comps:
        c = np.asarray(ua, dtype=float) - u
        c2 = c @ c
        P += ra * (Ta * np.eye(3) + np.outer(c, c))
        q += ra * c * (c2 + 5 * Ta)
        R += ra * (c2 * c2 + 10 * Ta * c2 + 15 * Ta * Ta)
    return np.array([rho, *u, P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2], *q, R])


def jets_like_field(nx: int, ny: int, setup: dict, spread=0.35, reach=0.8, rng=None,
                    uz_beam: float = 0.0):
    """A synthetic, developed-looking crossed-jets state on [0,1]^2: background
    gas plus two Maxwellian beams (the inflow states) whose densities decay
    away from the slots and spread with distance, so that the crossing
    region holds bimodal (strongly non-equilibrium) states.  Vectorised over
    cells: returns (ny, nx, 14) primitives."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    lo, hi = setup["slot"]
    yc, hw = 0.5 * (lo + hi), 0.5 * (hi - lo)
    jitter = 0.0 if rng is None else rng.uniform(-0.02, 0.02)

    def beam(s, n):        # s: distance along the jet, n: transverse offset
        w = hw + spread * s
        prof = 0.5 * (1 - np.tanh((np.abs(n) - w) / (0.01 + 0.05 * s)))
        return prof * (hw / w) * 0.5 * (1 - np.tanh((s - reach - jitter) / 0.05))

    rb = setup["background"][0]
    Tb = setup["background"][4] / rb
    rj = setup["left"][0]
    Tj = setup["left"][4] / rj
    ux = setup["left"][1]
    uy = setup["bottom"][2]
    w1 = rj * beam(X, Y - yc)
    w2 = rj * beam(Y, X - yc)
    # vectorised mixture of three Maxwellians
    comps = [(np.full_like(X, rb), (0.0, 0.0, 0.0), Tb), (w1 + 1e-30, (ux, 0.0, uz_beam), Tj),
             (w2 + 1e-30, (0.0, uy, 0.0), Tj)]
    rho = sum(c[0] for c in comps)
    u = [sum(c[0] * c[1][d] for c in comps) / rho for d in range(3)]
    out = np.zeros((ny, nx, 14))
    out[..., 0] = rho
    out[..., 1], out[..., 2], out[..., 3] = u
    P = [[0.0] * 3 for _ in range(3)]
    q = [0.0] * 3
    R = 0.0
    for ra, ua, Ta in comps:
        c = [ua[d] - u[d] for d in range(3)]
        c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2]
        for i in range(3):
            for j in range(3):
                P[i][j] = P[i][j] + ra * ((Ta if i == j else 0.0) + c[i] * c[j])
            q[i] = q[i] + ra * c[i] * (c2 + 5 * Ta)
        R = R + ra * (c2 * c2 + 10 * Ta * c2 + 15 * Ta * Ta)
    out[..., 4], out[..., 5], out[..., 6] = P[0][0], P[0][1], P[0][2]
    out[..., 7], out[..., 8], out[..., 9] = P[1][1], P[1][2], P[2][2]
    out[..., 10], out[..., 11], out[..., 12], out[..., 13] = q[0], q[1], q[2], R
    if uz_beam == 0.0:        # exact zeros for the z-odd moments of a planar state
        out[..., 3] = 0.0
        out[..., 6] = 0.0
        out[..., 8] = 0.0
        out[..., 12] = 0.0
    return out
