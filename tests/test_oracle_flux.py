"""Pins of the oracle's face fluxes (Sec. 3.1), first-order residuals on a
periodic 1D grid of random particle-cloud states (5- and 14-moment):

  * HLL upwinds a supersonic flow: when every wave speed of both neighbours
    is positive (S_L >= 0) the face flux is the left state's physical flux,
    so the residual of cell i is -(F(Q_i) - F(Q_{i-1}))/dx with F the point
    flux (itself pinned against particle sums).  The flow is made supersonic
    by a uniform velocity shift, which moves every wave speed by the same
    amount and leaves the central moments unchanged;
  * HLL equals Rusanov where the Davis speeds are symmetric: for states that
    are mirror-symmetric in x (u_x, P_xy, P_xz, q_x zero: clouds averaged with
    their x-mirror) lambda_min = -lambda_max (Sec. 5.1), so S_L = -S_R = a and
    both fluxes reduce to (F_L + F_R)/2 - a (U_R - U_L)/2; with a drift the
    two differ (the check is not vacuous)."""
import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore")
M = 4
SIG_LIM = 1e-4


def residual(orc, system, Q, flux):
    n = Q.shape[0]
    Qb = np.concatenate([Q[-M:], Q, Q[:M]])[None]
    cfg = orc.make_cfg(system=system, nx=n, ny=1, order=1, flux=flux, tau_model=0,
                       sigma_lim=SIG_LIM, sides=[{"type": 1}] * 4)
    return orc.block_residual(cfg, 0, 0, n, 1, orc.prim2cons_field(Qb))[0]


def clouds(system, rng, n, mirror=False):
    out = []
    for _ in range(n):
        nb = rng.integers(1, 4)
        ws, vs = [], []
        for _b in range(nb):
            w = rng.uniform(0.2, 1.0, 48) * rng.uniform(0.2, 1.0)
            if system == 5:
                v = rng.normal(rng.normal(0, 1), np.exp(rng.normal(0, 0.5)), 48)
            else:
                L = np.diag(np.exp(rng.normal(0, 0.5, 3)))
                Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
                v = rng.normal(size=(48, 3)) @ (Rm @ L).T + rng.normal(0, 1, 3)
            ws.append(w)
            vs.append(v)
        w, v = np.concatenate(ws) * rng.uniform(0.05, 2.0), np.concatenate(vs)
        if mirror:
            w = np.concatenate([w, w])
            v = np.concatenate([v, -v]) if system == 5 else np.concatenate([v, v * [-1, 1, 1]])
        out.append(wl.particle_moments5(w, v) if system == 5 else wl.particle_moments14(w, v))
    return np.array(out)


@pytest.mark.parametrize("system", [5, 14])
def test_hll_upwinds_supersonic_flow(orc, system):
    rng = np.random.default_rng(101 + system)
    n = 24
    Q = clouds(system, rng, n)
    Q[:, 1] = 0.0
    lo = np.array([orc.wavespeeds(q, SIG_LIM)[0] for q in Q])
    Q[:, 1] = -lo.min() + 0.5                      # every lambda_min >= 0.5
    assert min(orc.wavespeeds(q, SIG_LIM)[0] for q in Q) > 0.4
    F = np.array([orc.flux(q, SIG_LIM) for q in Q])
    expect = -(F - np.roll(F, 1, axis=0)) * n
    got = residual(orc, system, Q, orc.FLUX_HLL)
    scale = np.abs(F).max(axis=0) * n
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13 * scale.max())
    # Rusanov adds dissipation even here: it does not upwind
    rus = residual(orc, system, Q, orc.FLUX_RUSANOV)
    assert np.abs(rus - expect).max() > 1e-3 * scale.max()


@pytest.mark.parametrize("system", [5, 14])
def test_hll_equals_rusanov_for_mirror_symmetric_states(orc, system):
    rng = np.random.default_rng(202 + system)
    n = 24
    Q = clouds(system, rng, n, mirror=True)
    odd = [1, 3] if system == 5 else [1, 5, 6, 10]
    assert np.abs(Q[:, odd]).max() < 1e-12 * np.abs(Q).max()
    Q[:, odd] = 0.0
    for q in Q:
        lo, hi = orc.wavespeeds(q, SIG_LIM)
        assert lo == pytest.approx(-hi, rel=1e-12)
    h = residual(orc, system, Q, orc.FLUX_HLL)
    r = residual(orc, system, Q, orc.FLUX_RUSANOV)
    scale = np.abs(h).max()
    np.testing.assert_allclose(h, r, rtol=0, atol=1e-12 * scale)
    # with a drift the Davis speeds are no longer symmetric and the fluxes differ
    Q[:, 1] = 0.7
    h = residual(orc, system, Q, orc.FLUX_HLL)
    r = residual(orc, system, Q, orc.FLUX_RUSANOV)
    assert np.abs(h - r).max() > 1e-3 * np.abs(h).max()
