"""Pins of the FP64 oracle's point functions against facts the paper and the
mathematics fix (CPU only).

Each test names what it pins.  Independent routes used:
  * particle clouds: conserved densities and fluxes are plain sums
    sum_p w_p v_k psi(v_p) for any distribution whose closing moments are
    taken from the same cloud (Sec. 2.1 moment definitions);
  * Gauss-Hermite quadrature of a Maxwellian / anisotropic Gaussian (exact
    for the polynomial degrees involved);
  * closed forms derived by hand: realizability boundary (sigma = 1), the
    Gaussian/Junk end point (sigma = 0), the isotropic (Grad-like) limit,
    the 1D1V reduction of the 14-moment closure, the linearised 5-moment
    system at equilibrium.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from paper_2401_15233_gb300 import workloads as wl

SIG_LIM = 1e-4


def read_golden(name):
    """key = value lines of tests/golden/<name>; '#' starts a comment"""
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = line.split("=")
            out[k.strip()] = v.strip()
    return out


def psi14(v):
    """collision invariants and moment generators of the 14 conserved densities"""
    v2 = (v * v).sum(-1)
    out = [np.ones_like(v2), v[..., 0], v[..., 1], v[..., 2]]
    for i in range(3):
        for j in range(i, 3):
            out.append(v[..., i] * v[..., j])
    for i in range(3):
        out.append(v[..., i] * v2)
    out.append(v2 * v2)
    return np.stack(out, -1)


def psi5(v):
    return np.stack([v ** 0, v, v ** 2, v ** 3, v ** 4], -1)


def cloud14(rng, n=40):
    w = rng.uniform(0.1, 1.0, n)
    v = rng.normal(size=(n, 3)) @ rng.normal(size=(3, 3)) + rng.normal(0, 1, 3)
    return w, v


def cloud_closing14(w, v):
    Q = wl.particle_moments14(w, v)
    u = np.array(Q[1:4])
    c = v - u
    c2 = (c * c).sum(1)
    Qt = np.einsum("p,pi,pj,pk->ijk", w, c, c, c)
    Rt = np.einsum("p,pi,pj,p->ij", w, c, c, c2)
    S = np.einsum("p,pi,p->i", w, c, c2 * c2)
    return Q, Qt, Rt, S


def gauss_cloud3(rho, u, Pmat, n=7):
    """Quadrature 'particles' of an anisotropic Gaussian with covariance P/rho:
    exact for moments up to degree 2n-1."""
    x, wq = hermegauss(n)
    wq = wq / math.sqrt(2 * math.pi)
    L = np.linalg.cholesky(np.asarray(Pmat) / rho)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    W = np.einsum("a,b,c->abc", wq, wq, wq).reshape(-1) * rho
    return W, X @ L.T + np.asarray(u)


def P_of(Q):
    return np.array([[Q[4], Q[5], Q[6]], [Q[5], Q[7], Q[8]], [Q[6], Q[8], Q[9]]])


# --------------------------------------------------------------- a2: prim <-> cons
def test_roundtrip_prim_cons(orc):
    rng = np.random.default_rng(1)
    for Q in wl.random_prim14(rng, 50):
        Q2 = orc.cons2prim(orc.prim2cons(Q))
        scale = np.array([Q[0]] + [1] * 3 + [Q[4]] * 6 + [abs(Q[10:13]).max() + 1e-3] * 3 + [Q[13]])
        np.testing.assert_allclose(Q2, Q, rtol=0, atol=1e-12 * scale.max() * 10)
        assert np.all(abs(Q2 - Q) <= 1e-11 * (abs(Q) + scale))
    for Q in wl.random_prim5(rng, 50):
        Q2 = orc.cons2prim(orc.prim2cons(Q))
        assert np.all(abs(Q2 - Q) <= 1e-11 * (abs(Q) + abs(Q).max()))


def test_conserved_equal_particle_sums(orc):
    """a2 pinned: prim2cons(moments of a cloud) = sum_p w psi(v_p)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        w, v = cloud14(rng)
        Q = wl.particle_moments14(w, v)
        U = (w[:, None] * psi14(v)).sum(0)
        np.testing.assert_allclose(orc.prim2cons(Q), U, rtol=1e-12, atol=1e-12 * abs(U).max())
        w1 = rng.uniform(0.1, 1, 30); v1 = rng.normal(rng.normal(), 1.3, 30)
        Q5 = wl.particle_moments5(w1, v1)
        U5 = (w1[:, None] * psi5(v1)).sum(0)
        np.testing.assert_allclose(orc.prim2cons(Q5), U5, rtol=1e-12, atol=1e-12 * abs(U5).max())


# --------------------------------------------------------------- a6: physical flux
@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux14_given_closure_equals_particle_flux(orc, d):
    """a6 pinned: with the cloud's own closing moments, the printed k-fluxes
    equal <v_k psi f> summed over the cloud."""
    rng = np.random.default_rng(10 + d)
    for _ in range(20):
        w, v = cloud14(rng)
        Q, Qt, Rt, S = cloud_closing14(w, v)
        Fp = (w[:, None] * v[:, d:d + 1] * psi14(v)).sum(0)
        F = orc.flux14_given_closure(Q, Qt, Rt, S, d)
        np.testing.assert_allclose(F, Fp, rtol=1e-11, atol=1e-11 * abs(Fp).max())


def test_flux5_given_s_equals_particle_flux(orc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        w = rng.uniform(0.1, 1, 30); v = rng.normal(rng.normal(), 1.2, 30)
        Q = wl.particle_moments5(w, v)
        s = (w * (v - Q[1]) ** 5).sum()
        Fp = (w[:, None] * v[:, None] * psi5(v)).sum(0)
        np.testing.assert_allclose(orc.flux5_given_s(Q, s), Fp, rtol=1e-11,
                                   atol=1e-11 * abs(Fp).max())


# --------------------------------------------------------------- a9: BGK source
def test_bgk_source14_equals_maxwellian_moment_difference(orc):
    """a9 pinned: C = -(<psi f> - <psi M>)/tau with <psi M> by Gauss-Hermite."""
    rng = np.random.default_rng(3)
    tau = 0.37
    for _ in range(10):
        w, v = cloud14(rng)
        Q = wl.particle_moments14(w, v)
        U = (w[:, None] * psi14(v)).sum(0)
        T = (Q[4] + Q[7] + Q[9]) / (3 * Q[0])
        Wm, Vm = gauss_cloud3(Q[0], Q[1:4], np.eye(3) * Q[0] * T)
        UM = (Wm[:, None] * psi14(Vm)).sum(0)
        np.testing.assert_allclose(orc.source(Q, tau), -(U - UM) / tau, rtol=1e-10,
                                   atol=1e-10 * abs(U).max() / tau)


def test_bgk_source5_equals_maxwellian_moment_difference(orc):
    rng = np.random.default_rng(4)
    x, wq = hermegauss(8)
    wq = wq / math.sqrt(2 * math.pi)
    for _ in range(10):
        w = rng.uniform(0.1, 1, 30); v = rng.normal(rng.normal(), 1.2, 30)
        Q = wl.particle_moments5(w, v)
        U = (w[:, None] * psi5(v)).sum(0)
        vm = Q[1] + math.sqrt(Q[2] / Q[0]) * x
        UM = (Q[0] * wq[:, None] * psi5(vm)).sum(0)
        np.testing.assert_allclose(orc.source(Q, 0.5), -(U - UM) / 0.5, rtol=1e-10,
                                   atol=1e-10 * abs(U).max())


# --------------------------------------------------------------- a4: sigma
def test_sigma5_worked_value_and_special_lines(orc):
    # q* = 1/2, r* = 4: sigma = (sqrt(3) - 1)/4 (closed form of Eq. sigma-mapping-5mom)
    assert orc.sigma([1, 0, 1, 0.5, 4.0]) == pytest.approx((math.sqrt(3) - 1) / 4, rel=1e-14)
    # Maxwellian: sigma = 0 (end point of the Junk line)
    assert abs(orc.sigma(wl.maxwellian5(2.0, 0.3, 1.7))) < 1e-15
    # symmetric state below Gaussian kurtosis: uniform distribution, r* = 9/5 -> sigma = (3-r*)/2
    a = 1.3
    Q = [1.0, 0.0, a * a / 3, 0.0, a ** 4 / 5]
    assert orc.sigma(Q) == pytest.approx(0.6, rel=1e-13)


def test_sigma5_is_one_on_realizability_boundary(orc):
    """Two-point distributions saturate r* >= q*^2 + 1 (Hamburger) -> sigma = 1."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        w = rng.uniform(0.05, 1, 2); v = rng.normal(0, 2, 2)
        Q = wl.particle_moments5(w, v)
        assert orc.sigma(Q) == pytest.approx(1.0, abs=1e-9)


def test_sigma5_identity_r_from_sigma(orc):
    """Eq. (sigma-mapping-5mom) inverts to r* = 3 - 2 sigma + q*^2/sigma."""
    rng = np.random.default_rng(7)
    for Q in wl.random_prim5(rng, 40):
        th = Q[2] / Q[0]
        qs = Q[3] / (Q[0] * th ** 1.5); rs = Q[4] / (Q[0] * th * th)
        s = orc.sigma(Q)
        if s > 1e-6 and abs(qs) > 1e-6:
            assert 3 - 2 * s + qs * qs / s == pytest.approx(rs, rel=1e-10)


def test_sigma14_is_one_on_sphere_distributions(orc):
    """Clouds on a sphere in velocity space saturate the realizability bound
    of Eq. (phys-realizability-3D3Vgas) -> sigma = 1."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        n = 30
        d = rng.normal(size=(n, 3)); d /= np.linalg.norm(d, axis=1)[:, None]
        v = rng.normal(0, 1, 3) + rng.uniform(0.5, 2) * d
        w = rng.uniform(0.1, 1, n)
        assert orc.sigma(wl.particle_moments14(w, v)) == pytest.approx(1.0, abs=1e-9)


def test_sigma14_is_zero_at_any_gaussian(orc):
    rng = np.random.default_rng(9)
    for _ in range(10):
        A = rng.normal(size=(3, 3)); Pm = A @ A.T + 0.3 * np.eye(3)
        W, V = gauss_cloud3(rng.uniform(0.1, 2), rng.normal(0, 1, 3), Pm)
        Q = wl.particle_moments14(W, V)
        assert abs(orc.sigma(Q)) < 1e-7


def test_sigma14_realizable_clouds_in_unit_interval(orc):
    rng = np.random.default_rng(11)
    for Q in wl.random_prim14(rng, 60):
        s = orc.sigma(Q)
        assert -1e-12 <= s <= 1 + 1e-9


# --------------------------------------------------------------- a5: closure
def test_closure14_trace_identities(orc):
    """K contracts to the identity: Q_ijj = q_i; unclamped sigma gives
    R_iikk = R_iijj (Eqs. closure-14mom-Qijk/Rijkk with Eq. sigma-mapping-14mom)."""
    rng = np.random.default_rng(12)
    for Q in wl.random_prim14(rng, 60):
        Qt, Rt, S = orc.closure14(Q, 1e-300)
        np.testing.assert_allclose(np.einsum("ijj->i", Qt), Q[10:13], rtol=1e-10,
                                   atol=1e-10 * (abs(Q[10:13]).max() + Q[0] * ((Q[4] + Q[7] + Q[9]) / 3 / Q[0]) ** 1.5))
        # full symmetry of Q_ijk and R_ijkk
        for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0)]:
            np.testing.assert_allclose(Qt, Qt.transpose(perm), rtol=1e-12, atol=1e-12 * abs(Qt).max())
        np.testing.assert_allclose(Rt, Rt.T, rtol=1e-12, atol=1e-12 * abs(Rt).max())
        s = orc.sigma(Q)
        if 1e-6 < s < 1.0:
            assert np.trace(Rt) == pytest.approx(Q[13], rel=1e-9)


def test_closure14_isotropic_grad_limit(orc):
    """Isotropic P = p I: Q_ijk = (d_jk q_i + d_ik q_j + d_ij q_k)/5,
    R_ijkk = (2 q_i q_j + d_ij |q|^2)/(5 sigma p) + (5 - 2 sigma) p^2 d_ij / rho,
    S_i = 3|q|^2 q_i/(5 sigma^2 p^2) + (14 - 8 sqrt(sigma)) (p/rho) q_i."""
    rng = np.random.default_rng(13)
    for _ in range(20):
        rho, p = rng.uniform(0.2, 2), rng.uniform(0.2, 2)
        q = rng.normal(0, 0.3, 3) * rho * (p / rho) ** 1.5
        R = rng.uniform(1.0, 1.4) * 15 * p * p / rho
        Q = np.array([rho, 0.1, -0.2, 0.3, p, 0, 0, p, 0, p, *q, R])
        sb = min(max(orc.sigma(Q), SIG_LIM), 1.0)
        Qt, Rt, S = orc.closure14(Q, SIG_LIM)
        I = np.eye(3)
        Qe = (np.einsum("jk,i->ijk", I, q) + np.einsum("ik,j->ijk", I, q) + np.einsum("ij,k->ijk", I, q)) / 5
        np.testing.assert_allclose(Qt, Qe, rtol=1e-11, atol=1e-12 * abs(q).max())
        q2 = q @ q
        Re = (2 * np.outer(q, q) + I * q2) / (5 * sb * p) + (5 - 2 * sb) * p * p * I / rho
        np.testing.assert_allclose(Rt, Re, rtol=1e-10, atol=1e-12 * abs(Re).max())
        Se = 3 * q2 * q / (5 * sb * sb * p * p) + (14 - 8 * math.sqrt(sb)) * (p / rho) * q
        np.testing.assert_allclose(S, Se, rtol=1e-9, atol=1e-12 * abs(Se).max())


def test_closure14_reduces_to_5moment_in_1d1v_limit(orc):
    """P = diag(p, e, e), q = (q, 0, 0), e -> 0: the 14-moment closure
    collapses to the 5-moment closure (Appendix B remark): S_x -> s,
    Q_xxx -> q, R_xxkk -> r, with the same sigma."""
    rng = np.random.default_rng(14)
    for _ in range(20):
        rho, p = rng.uniform(0.3, 2), rng.uniform(0.3, 2)
        th = p / rho
        qs = rng.normal(0, 0.8)
        sig_target = rng.uniform(0.01, 0.9)
        rs = 3 - 2 * sig_target + qs * qs / sig_target
        q = qs * rho * th ** 1.5
        r = rs * rho * th * th
        Q5 = np.array([rho, 0.2, p, q, r])
        e = 1e-9 * p
        # R_iijj of the 3D state -> r as e -> 0 (transverse energy is O(e))
        Q14 = np.array([rho, 0.2, 0, 0, p, 0, 0, e, 0, e, q, 0, 0, r])
        assert orc.sigma(Q14) == pytest.approx(orc.sigma(Q5), rel=1e-6)
        Qt, Rt, S = orc.closure14(Q14, SIG_LIM)
        s5 = orc.closure5(Q5, SIG_LIM)
        assert Qt[0, 0, 0] == pytest.approx(q, rel=1e-6)
        assert Rt[0, 0] == pytest.approx(r, rel=1e-6)
        assert S[0] == pytest.approx(s5, rel=1e-6, abs=1e-9 * abs(rho * th ** 2.5))


def test_closure14_rotation_covariance(orc):
    rng = np.random.default_rng(15)
    for Q in wl.random_prim14(rng, 20):
        Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        P = P_of(Q)
        P2 = Rm @ P @ Rm.T
        q2 = Rm @ Q[10:13]
        u2 = Rm @ Q[1:4]
        Qr = np.array([Q[0], *u2, P2[0, 0], P2[0, 1], P2[0, 2], P2[1, 1], P2[1, 2], P2[2, 2], *q2, Q[13]])
        Qt, Rt, S = orc.closure14(Q, SIG_LIM)
        Qt2, Rt2, S2 = orc.closure14(Qr, SIG_LIM)
        sc = abs(Qt).max() + 1e-30
        np.testing.assert_allclose(Qt2, np.einsum("ia,jb,kc,abc->ijk", Rm, Rm, Rm, Qt), atol=1e-9 * sc)
        np.testing.assert_allclose(Rt2, Rm @ Rt @ Rm.T, atol=1e-9 * abs(Rt).max())
        np.testing.assert_allclose(S2, Rm @ S, atol=1e-8 * (abs(S).max() + 1e-30))


def test_closure14_gaussian_limit_is_isserlis(orc):
    """q = 0 at the Gaussian kurtosis: sigma = 0 -> sigma_bar = sigma_lim,
    Q = 0, S = 0 and R_ijkk -> <c_i c_j c^2> of the Gaussian (Isserlis) as
    sigma_lim -> 0."""
    rng = np.random.default_rng(16)
    for _ in range(10):
        A = rng.normal(size=(3, 3)); Pm = A @ A.T + 0.3 * np.eye(3)
        W, V = gauss_cloud3(rng.uniform(0.1, 2), rng.normal(0, 1, 3), Pm)
        Q, Qg, Rg, Sg = cloud_closing14(W, V)
        Q[10:13] = 0.0
        Qt, Rt, S = orc.closure14(Q, 1e-12)
        assert abs(Qt).max() == 0.0 and abs(S).max() == 0.0
        np.testing.assert_allclose(Rt, Rg, rtol=1e-9, atol=1e-9 * abs(Rg).max())


def test_closure5_worked_value(orc):
    # q* = 1/2, r* = 4  ->  s* = q*^3/sigma^2 + (10 - 8 sigma^(1/2)) q*
    golden = read_golden("closure5_worked.txt")
    assert orc.closure5([1, 0, 1, 0.5, 4.0], 1e-4) == pytest.approx(float(golden["s_star"]), rel=1e-9)


# --------------------------------------------------------------- a7: wave speeds
def test_baradaran_special_values(orc):
    """Eq. (ws-max-baradaran-orig): lambda* = 1 at q* = 0 on the realizability
    boundary (sigma = 1); lambda* -> sqrt(5 + sqrt(10)) (Grad-5 speed) as
    sigma -> 0 at q* = 0."""
    assert orc.lambda_star5(0.0, 1.0) == pytest.approx(1.0, rel=1e-15)
    assert orc.lambda_star5(0.0, 1e-16) == pytest.approx(math.sqrt(5 + math.sqrt(10)), rel=1e-7)


def test_ws14_closed_forms_at_isotropic_rest(orc):
    """At P*_xx = 1, q* = 0 the bracket is 2 sigma |sqrt(B) - E| so
    lambda* = (a sigma + b)|sqrt(B) - E| + E with a = 1.4/e, b = 0.9/sqrt(e).
    sigma = 1: lambda* = a + b.  sigma -> 0: b (sqrt(5 + sqrt 10) - 0.8 sqrt 3) + 0.8 sqrt 3."""
    a, b = 1.4 * math.exp(-1), 0.9 * math.exp(-0.5)
    assert orc.lambda_star14(1.0, 0.0, 0.0, 1.0) == pytest.approx(a + b, rel=1e-14)
    g0 = b * (math.sqrt(5 + math.sqrt(10)) - 0.8 * math.sqrt(3)) + 0.8 * math.sqrt(3)
    assert orc.lambda_star14(1.0, 0.0, 0.0, 1e-16) == pytest.approx(g0, rel=1e-7)
    golden = read_golden("ws14_worked.txt")
    assert orc.lambda_star14(1.0, 0.0, 0.0, 1e-4) == pytest.approx(float(golden["lam_q0_s1e-4"]), rel=1e-7)
    assert orc.lambda_star14(1.0, 0.5, 0.0, 1e-4) == pytest.approx(float(golden["lam_max_qx05_s1e-4"]), rel=1e-7)
    assert -orc.lambda_star14(1.0, -0.5, 0.0, 1e-4) == pytest.approx(float(golden["lam_min_qx05_s1e-4"]), rel=1e-7)


def _mirror_x(Q):
    Q = np.array(Q, dtype=float)
    for k in (1, 5, 6, 10):       # u_x, P_xy, P_xz, q_x
        Q[k] = -Q[k]
    return Q


def _swap_xy(Q):
    Q = np.array(Q, dtype=float)
    return Q[[0, 2, 1, 3, 7, 5, 8, 4, 6, 9, 11, 10, 12, 13]]


def test_ws14_symmetries(orc):
    """lambda_min(Q) = -lambda_max(mirror_x Q) (Sec. 5.1); y-speeds equal
    x-speeds of the x<->y transposed state; rotation about x leaves the
    x-speeds unchanged; lambda_max > u_x > lambda_min."""
    rng = np.random.default_rng(17)
    for Q in wl.random_prim14(rng, 40):
        lo, hi = orc.wavespeeds(Q, SIG_LIM, 1.0, 0)
        lo2, hi2 = orc.wavespeeds(_mirror_x(Q), SIG_LIM, 1.0, 0)
        assert lo == pytest.approx(-hi2, rel=1e-12, abs=1e-12)
        assert hi > Q[1] > lo
        ylo, yhi = orc.wavespeeds(Q, SIG_LIM, 1.0, 1)
        xlo, xhi = orc.wavespeeds(_swap_xy(Q), SIG_LIM, 1.0, 0)
        assert (ylo, yhi) == pytest.approx((xlo, xhi), rel=1e-12, abs=1e-12)
        th = rng.uniform(0, 2 * np.pi)
        Rm = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
        P2 = Rm @ P_of(Q) @ Rm.T
        Qr = np.array([Q[0], *(Rm @ Q[1:4]), P2[0, 0], P2[0, 1], P2[0, 2], P2[1, 1], P2[1, 2],
                       P2[2, 2], *(Rm @ Q[10:13]), Q[13]])
        assert orc.wavespeeds(Qr, SIG_LIM, 1.0, 0) == pytest.approx((lo, hi), rel=1e-11, abs=1e-11)


def test_flux5_jacobian_at_equilibrium_matches_linear_theory(orc):
    """Linearising Eq. (5mom-sys-eqs) with the closure at a Maxwellian gives
    s = alpha q (alpha = 10 - 8 sqrt(sigma_lim)) and characteristic speeds
    u + c * {0, +-sqrt((alpha +- sqrt(alpha^2 - 12 alpha + 60))/2)}.
    The finite-difference Jacobian of the oracle's flux must reproduce them;
    at sigma_lim -> 0 the largest is the Grad-5 speed that the Baradaran fit
    also returns."""
    for (rho, u, T) in [(1.0, 0.0, 1.0), (0.3, 1.7, 2.5)]:
        Q = wl.maxwellian5(rho, u, T)
        U0 = orc.prim2cons(Q)
        J = np.zeros((5, 5))
        for k in range(5):
            h = 1e-8 * max(abs(U0[k]), 1.0)   # h << sigma_lim keeps q^3/sigma^2 out
            Up = U0.copy(); Up[k] += h
            Um = U0.copy(); Um[k] -= h
            J[:, k] = (orc.flux(orc.cons2prim(Up), SIG_LIM) - orc.flux(orc.cons2prim(Um), SIG_LIM)) / (2 * h)
        ev = np.sort(np.linalg.eigvals(J).real)
        al = 10 - 8 * math.sqrt(SIG_LIM)
        r = math.sqrt(al * al - 12 * al + 60)
        c = math.sqrt(T)
        exp_ev = np.sort(u + c * np.array([0, math.sqrt((al + r) / 2), -math.sqrt((al + r) / 2),
                                           math.sqrt((al - r) / 2), -math.sqrt((al - r) / 2)]))
        np.testing.assert_allclose(ev, exp_ev, atol=1e-6 * (abs(u) + c))


def test_ws14_transverse_heat_flux_terms(orc):
    """Transverse terms of Eq. (14mom-approx-ws-equations) at sigma = 1,
    P*_xx = 1, q*_x = 0, |q*_perp| = 1: E = C = 0, B = Y = 1,
    zeta = 0.6 - 0.38 + 0.35 = 0.57, so
    lambda* = ((a + b)/2) (0.57 + sqrt(0.57^2 + 4 + 1/10))."""
    a, b = 1.4 * math.exp(-1), 0.9 * math.exp(-0.5)
    want = 0.5 * (a + b) * (0.57 + math.sqrt(0.57 ** 2 + 4.1))
    assert orc.lambda_star14(1.0, 0.0, 1.0, 1.0) == pytest.approx(want, rel=1e-14)
    # anisotropic P*_xx = 2, sigma = 1: a = 1.4 2^1.1 e^-4, b = 1.8 exp(-2^1.4/2)
    a2, b2 = 1.4 * 2 ** 1.1 * math.exp(-4), 1.8 * math.exp(-0.5 * 2 ** 1.4)
    z = 0.3 + 0.5 * (0.6 * 4 - 0.76 + 0.35)
    want2 = 0.5 * (a2 + b2) * (z + math.sqrt(z * z + 4 + 0.025))
    assert orc.lambda_star14(2.0, 0.3, 0.5, 1.0) == pytest.approx(want2, rel=1e-14)


# ------------------------------------------- a7: 5-moment fit away from q* = 0
def test_baradaran_worked_values_off_axis(orc):
    """Eq. (ws-max-baradaran-orig) at sigma = 1e-4, q* = +-1/2, against the
    hand evaluation in tests/golden/ws5_worked.txt.  The q* < 0 value comes
    from the rationalised bracket (reading: no cancellation) and also pins
    lambda*_min(q*) = -lambda*_max(-q*) through the re-dimensionalised
    speeds of a state with that q*."""
    g = read_golden("ws5_worked.txt")
    assert orc.lambda_star5(0.5, 1e-4) == pytest.approx(float(g["lam_max_q+05_s1e-4"]), rel=1e-13)
    assert orc.lambda_star5(-0.5, 1e-4) == pytest.approx(float(g["lam_max_q-05_s1e-4"]), rel=1e-13)
    # a state with rho = 2, u = 0.3, P = 8 (theta = 4), q* = 1/2 and the sigma
    # of r* chosen so that sigma = 1e-4 exactly in real arithmetic:
    # r* = 3 - 2 sigma + q*^2/sigma (Eq. sigma-mapping-5mom inverted)
    rho, u, th, qs, sg = 2.0, 0.3, 4.0, 0.5, 1e-4
    rs = 3 - 2 * sg + qs * qs / sg
    Q = [rho, u, rho * th, qs * rho * th ** 1.5, rs * rho * th * th]
    lo, hi = orc.wavespeeds(Q, 1e-6, 1.0)
    assert hi == pytest.approx(u + 2.0 * float(g["lam_max_q+05_s1e-4"]), rel=1e-9)
    assert lo == pytest.approx(u - 2.0 * float(g["lam_max_q-05_s1e-4"]), rel=1e-9)


def test_baradaran_on_realizability_boundary_is_two_delta_speed(orc):
    """At sigma = 1 the distribution is two delta functions (Sec. 2.3.1).
    With zero mean and unit variance their velocities c1 < 0 < c2 satisfy
    c1 c2 = -1 and c1 + c2 = q* (the third moment), so the fastest and
    slowest signals travel at (q* +- sqrt(q*^2 + 4))/2.  Eq.
    (ws-max-baradaran-orig) must return exactly these: C = E = 0 there, so
    this fixes the hyperbolic part (its 1/(2 sigma) factor, the sign of q*
    and the 4 sigma^2 Y term with Y = 1)."""
    for qs in (-3.0, -0.5, 0.0, 0.25, 2.0):
        r = math.sqrt(qs * qs + 4)
        assert orc.lambda_star5(qs, 1.0) == pytest.approx((qs + r) / 2, rel=1e-14)
        assert -orc.lambda_star5(-qs, 1.0) == pytest.approx((qs - r) / 2, rel=1e-14)
    # the same from a two-particle cloud, through the full speed routine
    for (w1, w2, v1, v2) in [(0.3, 0.7, -1.1, 2.4), (0.8, 0.2, 0.5, 3.0)]:
        m = wl.particle_moments5(np.array([w1, w2]), np.array([v1, v2]))
        lo, hi = orc.wavespeeds(m, 1e-4, 1.0)
        assert orc.sigma(m) == pytest.approx(1.0, abs=1e-12)
        assert hi == pytest.approx(v2, rel=1e-6)
        assert lo == pytest.approx(v1, rel=1e-6, abs=1e-6)


def test_baradaran_small_sigma_asymptotes(orc):
    """Closed-form limits of Eq. (ws-max-baradaran-orig) as sigma -> 0 at
    fixed q* != 0 (C -> sqrt 3, E -> 0.8 sqrt 3):
      q* > 0: the bracket is 2q* + D0/(2q*) + O(sigma^2), so
              lambda* - q*/sigma -> E - C/5 = (3/5) sqrt 3;
      q* < 0: the bracket is D0/(2|q*|) + O(sigma^2), so
              lambda* -> E + C/5 = sqrt 3.
    A dropped or sign-flipped (4/5) q* sigma C term moves the first limit to
    0.8 sqrt 3 or sqrt 3 and the second to 0.8 sqrt 3 or (3/5) sqrt 3.  At
    sigma = 1e-14 the unrationalised bracket for q* < 0 loses ~1e-3 to
    cancellation, so the second limit also pins the rationalised form."""
    r3 = math.sqrt(3.0)
    for qs in (0.5, 2.0):
        s = 1e-6
        assert orc.lambda_star5(qs, s) - qs / s == pytest.approx(0.6 * r3, rel=1e-4)
    for qs in (-0.5, -2.0):
        assert orc.lambda_star5(qs, 1e-14) == pytest.approx(r3, rel=1e-9)


# ----------------------------------------------------------- a9: tau model
@pytest.mark.parametrize("system", [5, 14])
def test_tau_follows_mean_free_path_over_thermal_speed(orc, system):
    """Sec. 4: tau = (n sigma_cs v_th)^-1 with v_th = sqrt(8 k_B T / (pi m));
    Kn = lambda_ref / L with lambda_ref = 1/(n_ref sigma_cs) (the jets'
    sqrt(2) in lambda cancels the same way, Sec. 6).  Units: m = k_B = 1,
    n = rho; T = P/rho (1D1V) or tr P/(3 rho) (3D3V).  The cross-section is
    recovered from Kn and tau evaluated from its definition at two states
    that differ from the reference in both rho and T (an anisotropic P for
    14 moments), against the oracle's tau_ref (rho_ref/rho) sqrt(T_ref/T)."""
    Kn, L, rho_ref, T_ref = 0.03, 0.1, 1.0, 1.5
    sig_cs = 1.0 / (Kn * L * rho_ref)
    vth = lambda T: math.sqrt(8.0 * T / math.pi)
    tau_def = lambda rho, T: 1.0 / (rho * sig_cs * vth(T))
    cfg = orc.make_cfg(system=system, nx=4, tau_model=orc.TAU_HARDSPHERE,
                       tau_ref=tau_def(rho_ref, T_ref), rho_ref=rho_ref, T_ref=T_ref)
    for rho, T in [(0.125, 0.8), (2.0, 3.0)]:
        if system == 5:
            Q = [rho, 0.7, rho * T, 0.1 * rho * T ** 1.5, 3.2 * rho * T * T]
        else:
            Q = list(wl.maxwellian14(rho, 0.4, -0.2, T))
            Q[4] += 0.3 * rho * T; Q[7] -= 0.1 * rho * T; Q[9] -= 0.2 * rho * T   # tr P kept
            Q[5] += 0.05 * rho * T
        assert orc.tau(cfg, np.array(Q, dtype=float)) == pytest.approx(tau_def(rho, T), rel=1e-14)
    # hand value: Kn = 0.01, L = 1, rho_ref = T_ref = 1 at rho = 0.125, T = 0.8:
    # tau = 0.01 / (0.125 * 1.42729929) = 0.0560499122
    cfg1 = orc.make_cfg(system=5, nx=4, tau_model=orc.TAU_HARDSPHERE,
                        tau_ref=wl.sod_tau_ref(0.01), rho_ref=1.0, T_ref=1.0)
    assert orc.tau(cfg1, np.array([0.125, 0.0, 0.1, 0.0, 0.24])) == pytest.approx(0.0560499122, rel=1e-9)


# ------------------------------------------------------- a11: CFL rate and dt
LAM14_ISO = 2.1825987   # lambda* of a Maxwellian (sigma clamped to 1e-4), ws14_worked.txt
LAM5_ISO = 2.8455181    # Baradaran at q* = 0, sigma = 1e-4 (design-survey hand evaluation)


def test_cfl_rate_and_dt_2d_by_hand(orc):
    """Reading 10: dt = CFL / max_cells sum_d max(|lmin_d|, |lmax_d|)/dx_d.
    Maxwellian cells (q = 0, sigma clamped to sigma_lim) have
    lmax/lmin = u_d +- lambda* sqrt(T), so each cell's rate is
    (|u_x| + lambda* sqrt T)/dx + (|u_y| + lambda* sqrt T)/dy.  The states
    are chosen so that the cell with the largest sum (B) differs from the
    cell with the largest single-direction term (A), and dx != dy; the last
    step is clipped to t_end."""
    g = read_golden("ws14_worked.txt")
    lam = float(g["lam_q0_s1e-4"])
    assert lam == LAM14_ISO
    nx, ny, dx, dy = 3, 2, 1.0 / 3.0, 1.0 / 2.0
    cells = {(0, 0): (1.0, 6.0, 0.0, 1.0),      # A: 3*8.18 + 2*2.18 = 28.9
             (1, 0): (0.5, 4.0, -6.0, 1.0),     # B: 3*6.18 + 2*8.18 = 34.9
             (2, 0): (1e-3, 0.0, 0.0, 4.0),
             (0, 1): (1.0, 0.0, 0.0, 1.0),
             (1, 1): (2.0, -1.0, 1.0, 0.25),
             (2, 1): (1.0, 0.5, 2.5, 1.0)}
    prim = np.zeros((ny, nx, 14))
    want = 0.0
    for (i, j), (rho, ux, uy, T) in cells.items():
        prim[j, i] = wl.maxwellian14(rho, ux, uy, T)
        r = (abs(ux) + lam * math.sqrt(T)) / dx + (abs(uy) + lam * math.sqrt(T)) / dy
        want = max(want, r)
    assert want == pytest.approx(3 * (4 + lam) + 2 * (6 + lam))   # cell B
    cfg = orc.make_cfg(system=14, nx=nx, ny=ny, cfl=0.5)
    U = orc.prim2cons_field(prim)
    assert orc.max_rate(cfg, U) == pytest.approx(want, rel=2e-7)
    dt_full = 0.5 / want
    assert orc.dt(cfg, U, 0.0, 10.0) == pytest.approx(dt_full, rel=2e-7)
    assert orc.dt(cfg, U, 1.0, 1.0 + 0.25 * dt_full) == pytest.approx(0.25 * dt_full, rel=1e-9)


def test_cfl_rate_and_dt_1d_by_hand(orc):
    """The same for the 5-moment tube: rate = (|u| + lambda* sqrt T)/dx with
    Baradaran's lambda*(q* = 0, sigma_lim = 1e-4)."""
    nx, dx = 4, 0.25
    cells = [(1.0, -3.0, 1.0), (0.2, 1.0, 4.0), (1.0, 0.0, 1.0), (0.125, 0.5, 0.8)]
    prim = np.array([wl.maxwellian5(*c) for c in cells])[None]
    want = max((abs(u) + LAM5_ISO * math.sqrt(T)) / dx for (_, u, T) in cells)
    assert want == pytest.approx(4 * (1 + 2 * LAM5_ISO))
    cfg = orc.make_cfg(system=5, nx=nx, ny=1, cfl=0.5)
    U = orc.prim2cons_field(prim)
    assert orc.max_rate(cfg, U) == pytest.approx(want, rel=2e-7)
    assert orc.dt(cfg, U, 0.0, 10.0) == pytest.approx(0.5 / want, rel=2e-7)
    assert orc.dt(cfg, U, 0.1, 0.1 + 1e-5) == pytest.approx(1e-5, rel=1e-9)
