"""Python access to the plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is the slow, literal C implementation in ``maxent_oracle.c`` of the
maximum-entropy 5- and 14-moment method (Boccelli et al., JCP 2024).  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "maxent_oracle.c")
_LIB = os.path.join(_HERE, "libmaxent_oracle.so")
_OMPLIB = os.path.join(_HERE, "libmaxent_oracle_omp.so")
_TSRC = os.path.join(_HERE, "tangent.cpp")
_TLIB = os.path.join(_HERE, "libmaxent_oracle_tangent.so")

BC_TRANSMISSIVE, BC_PERIODIC, BC_DIRICHLET = 0, 1, 2
FLUX_HLL, FLUX_RUSANOV = 0, 1
LIM_MINMOD, LIM_VANALBADA = 0, 1
TAU_NONE, TAU_CONST, TAU_HARDSPHERE = 0, 1, 2
FE, RK2 = 0, 1
SRC_EXPLICIT, SRC_POINT_IMPLICIT = 0, 1
MAX_SPANS = 4
MARGIN = 4


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction).  omp=True: the
    OpenMP timing build (same arithmetic, loops over rows and columns on
    all host cores; bitwise equal results)."""
    out = _OMPLIB if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "maxent_oracle.h"))
    ):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", out + ".tmp", _SRC, "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)
    return out


def build_tangent(force: bool = False) -> str:
    """Compile the forward-mode tangent: the same oracle source with a
    dual-number arithmetic type (g++, no FMA contraction)."""
    deps = [_SRC, _TSRC, os.path.join(_HERE, "maxent_oracle.h")]
    if force or not os.path.exists(_TLIB) or os.path.getmtime(_TLIB) < max(
            os.path.getmtime(d) for d in deps):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _TLIB + ".tmp", _TSRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_TLIB + ".tmp", _TLIB)
    return _TLIB


class Side(C.Structure):
    _fields_ = [
        ("base_type", C.c_int),
        ("base_state", C.c_double * 14),
        ("nspans", C.c_int),
        ("span_lo", C.c_double * MAX_SPANS),
        ("span_hi", C.c_double * MAX_SPANS),
        ("span_state", (C.c_double * 14) * MAX_SPANS),
    ]


class Cfg(C.Structure):
    _fields_ = [
        ("system", C.c_int),
        ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("order", C.c_int), ("integrator", C.c_int), ("flux", C.c_int), ("limiter", C.c_int),
        ("cfl", C.c_double), ("sigma_lim", C.c_double), ("k_ws", C.c_double),
        ("tau_model", C.c_int),
        ("tau_ref", C.c_double), ("rho_ref", C.c_double), ("T_ref", C.c_double),
        ("side", Side * 4),
        ("source_scheme", C.c_int),
        ("frozen_limiter", C.c_int),
    ]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


_omplib = None


def lib_omp():
    """The OpenMP timing build (thread count from OMP_NUM_THREADS, else all
    cores).  Same functions as lib()."""
    global _omplib
    if _omplib is None:
        _omplib = _declare(C.CDLL(build(omp=True)))
    return _omplib


def threads(omp: bool = False) -> int:
    """Threads the scheme loops of that build use."""
    return (lib_omp() if omp else lib()).or_threads()


def _declare(L):
    """argument and result types of the exported functions"""
    for name in ("or5_prim2cons", "or5_cons2prim", "or14_prim2cons", "or14_cons2prim"):
        getattr(L, name).argtypes = [_dp, _dp]
        getattr(L, name).restype = None
    L.or5_sigma.argtypes = [_dp]; L.or5_sigma.restype = C.c_double
    L.or14_sigma.argtypes = [_dp]; L.or14_sigma.restype = C.c_double
    L.or5_closure.argtypes = [_dp, C.c_double]; L.or5_closure.restype = C.c_double
    L.or5_flux_given_s.argtypes = [_dp, C.c_double, _dp]; L.or5_flux_given_s.restype = None
    L.or5_flux.argtypes = [_dp, C.c_double, _dp]; L.or5_flux.restype = None
    L.or5_lambda_star_max.argtypes = [C.c_double, C.c_double]
    L.or5_lambda_star_max.restype = C.c_double
    L.or5_wavespeeds.argtypes = [_dp, C.c_double, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.or5_wavespeeds.restype = None
    L.or5_source.argtypes = [_dp, C.c_double, _dp]; L.or5_source.restype = None
    L.or14_closure.argtypes = [_dp, C.c_double, _dp, _dp, _dp]
    L.or14_closure.restype = None
    L.or14_flux_given_closure.argtypes = [_dp, _dp, _dp, _dp, C.c_int, _dp]
    L.or14_flux_given_closure.restype = None
    L.or14_flux.argtypes = [_dp, C.c_double, C.c_int, _dp]; L.or14_flux.restype = None
    L.or14_lambda_star_max.argtypes = [C.c_double] * 4
    L.or14_lambda_star_max.restype = C.c_double
    L.or14_wavespeeds.argtypes = [_dp, C.c_int, C.c_double, C.c_double,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.or14_wavespeeds.restype = None
    L.or14_source.argtypes = [_dp, C.c_double, _dp]; L.or14_source.restype = None
    L.or_block_step.argtypes = [C.POINTER(Cfg), C.c_int, C.c_int, C.c_int, C.c_int,
                                _dp, C.c_double, _dp]
    L.or_block_step.restype = C.c_int
    L.or_block_residual.argtypes = [C.POINTER(Cfg), C.c_int, C.c_int, C.c_int, C.c_int,
                                    _dp, _dp]
    L.or_block_residual.restype = C.c_int
    L.or_max_rate.argtypes = [C.POINTER(Cfg), _dp]; L.or_max_rate.restype = C.c_double
    L.or_dt.argtypes = [C.POINTER(Cfg), _dp, C.c_double, C.c_double]
    L.or_dt.restype = C.c_double
    L.or_step.argtypes = [C.POINTER(Cfg), _dp, C.c_double]; L.or_step.restype = C.c_int
    L.or_run.argtypes = [C.POINTER(Cfg), _dp, C.POINTER(C.c_double), C.c_double,
                         C.c_int, C.c_void_p]
    L.or_run.restype = C.c_int
    L.or_tau.argtypes = [C.POINTER(Cfg), _dp]; L.or_tau.restype = C.c_double
    L.or_prim2cons_n.argtypes = [C.c_int, C.c_long, _dp, _dp]; L.or_prim2cons_n.restype = None
    L.or_cons2prim_n.argtypes = [C.c_int, C.c_long, _dp, _dp]; L.or_cons2prim_n.restype = None
    L.or_threads.argtypes = []; L.or_threads.restype = C.c_int
    return L


def _a(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.shape == (n,), a.shape
    return a


# ---------------------------------------------------------------- point API
def prim2cons(Q):
    Q = _a(Q); U = np.empty_like(Q)
    (lib().or5_prim2cons if Q.size == 5 else lib().or14_prim2cons)(Q, U)
    return U


def prim2cons_field(Q):
    """(..., nf) primitive field -> conserved, cell by cell"""
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    U = np.empty_like(Q)
    nf = Q.shape[-1]
    lib().or_prim2cons_n(nf, Q.size // nf, Q.reshape(-1), U.reshape(-1))
    return U


def cons2prim_field(U):
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    Q = np.empty_like(U)
    nf = U.shape[-1]
    lib().or_cons2prim_n(nf, U.size // nf, U.reshape(-1), Q.reshape(-1))
    return Q


def cons2prim(U):
    U = _a(U); Q = np.empty_like(U)
    (lib().or5_cons2prim if U.size == 5 else lib().or14_cons2prim)(U, Q)
    return Q


def sigma(Q):
    Q = _a(Q)
    return (lib().or5_sigma if Q.size == 5 else lib().or14_sigma)(Q)


def closure5(Q, sigma_lim):
    return lib().or5_closure(_a(Q, 5), sigma_lim)


def closure14(Q, sigma_lim):
    Qt = np.empty(27); Rt = np.empty(9); S = np.empty(3)
    lib().or14_closure(_a(Q, 14), sigma_lim, Qt, Rt, S)
    return Qt.reshape(3, 3, 3), Rt.reshape(3, 3), S


def flux5_given_s(Q, s):
    F = np.empty(5); lib().or5_flux_given_s(_a(Q, 5), s, F); return F


def flux14_given_closure(Q, Qt, Rt, S, d):
    F = np.empty(14)
    lib().or14_flux_given_closure(_a(Q, 14), _a(np.ravel(Qt), 27), _a(np.ravel(Rt), 9),
                                  _a(S, 3), d, F)
    return F


def flux(Q, sigma_lim, d=0):
    Q = _a(Q); F = np.empty_like(Q)
    if Q.size == 5:
        lib().or5_flux(Q, sigma_lim, F)
    else:
        lib().or14_flux(Q, sigma_lim, d, F)
    return F


def lambda_star5(qs, sig):
    return lib().or5_lambda_star_max(qs, sig)


def lambda_star14(Pdd, qd, qperp, sig):
    return lib().or14_lambda_star_max(Pdd, qd, qperp, sig)


def wavespeeds(Q, sigma_lim, k=1.0, d=0):
    Q = _a(Q); lo = C.c_double(); hi = C.c_double()
    if Q.size == 5:
        lib().or5_wavespeeds(Q, sigma_lim, k, C.byref(lo), C.byref(hi))
    else:
        lib().or14_wavespeeds(Q, d, sigma_lim, k, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def source(Q, tau):
    Q = _a(Q); Cv = np.empty_like(Q)
    (lib().or5_source if Q.size == 5 else lib().or14_source)(Q, tau, Cv)
    return Cv


# ---------------------------------------------------------------- scheme API
def make_cfg(system=14, nx=64, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, order=2,
             integrator=RK2, flux=FLUX_HLL, limiter=LIM_MINMOD, cfl=0.5,
             sigma_lim=1e-4, k_ws=1.0, tau_model=TAU_NONE, tau_ref=1.0, rho_ref=1.0,
             T_ref=1.0, sides=None, source_scheme=0) -> Cfg:
    """sides: list of 4 dicts {type, state (prim), spans: [(lo, hi, prim), ...]};
    source_scheme: SRC_EXPLICIT (BGK source in the stage residual) or
    SRC_POINT_IMPLICIT (backward-Euler relaxation after each stage)."""
    c = Cfg()
    c.system, c.nx, c.ny = system, nx, ny
    c.x0, c.x1, c.y0, c.y1 = x0, x1, y0, y1
    c.order, c.integrator, c.flux, c.limiter = order, integrator, flux, limiter
    c.cfl, c.sigma_lim, c.k_ws = cfl, sigma_lim, k_ws
    c.tau_model, c.tau_ref, c.rho_ref, c.T_ref = tau_model, tau_ref, rho_ref, T_ref
    c.source_scheme = source_scheme
    sides = sides or [{} for _ in range(4)]
    for s, sd in enumerate(sides):
        c.side[s].base_type = sd.get("type", BC_TRANSMISSIVE)
        st = sd.get("state")
        if st is not None:
            for k, v in enumerate(st):
                c.side[s].base_state[k] = v
        spans = sd.get("spans", [])
        assert len(spans) <= MAX_SPANS
        c.side[s].nspans = len(spans)
        for n, (lo, hi, prim) in enumerate(spans):
            c.side[s].span_lo[n] = lo
            c.side[s].span_hi[n] = hi
            for k, v in enumerate(prim):
                c.side[s].span_state[n][k] = v
    return c


def nf_of(cfg: Cfg) -> int:
    return 5 if cfg.system == 5 else 14


def max_rate(cfg: Cfg, U, omp=False):
    """U: (ny, nx, nf) conserved, interior cells."""
    return (lib_omp() if omp else lib()).or_max_rate(C.byref(cfg), _a(U).reshape(-1))


def dt(cfg: Cfg, U, t, t_end, omp=False):
    return (lib_omp() if omp else lib()).or_dt(C.byref(cfg), _a(U).reshape(-1), t, t_end)


def step(cfg: Cfg, U, dtv, omp=False):
    """Advance U (ny, nx, nf) by one step of size dt; returns a new array."""
    out = np.array(U, dtype=np.float64, order="C", copy=True)
    flat = out.reshape(-1)
    rc = (lib_omp() if omp else lib()).or_step(C.byref(cfg), flat, dtv)
    assert rc == 0
    return out


def run(cfg: Cfg, U, t, t_end, max_steps, omp=False):
    out = np.array(U, dtype=np.float64, order="C", copy=True)
    tt = C.c_double(t)
    hist = np.zeros(max(max_steps, 1))
    n = (lib_omp() if omp else lib()).or_run(C.byref(cfg), out.reshape(-1), C.byref(tt), t_end,
                                             max_steps, hist.ctypes.data_as(C.c_void_p))
    return out, tt.value, hist[:n]


def block_step(cfg: Cfg, i0, j0, w, h, Ub, dtv):
    """Ub: block with margins, shape (h+2My, w+2Mx, nf)."""
    nf = nf_of(cfg)
    out = np.empty((h, w, nf))
    rc = lib().or_block_step(C.byref(cfg), i0, j0, w, h, _a(Ub).reshape(-1), dtv,
                             out.reshape(-1))
    assert rc == 0
    return out


def block_residual(cfg: Cfg, i0, j0, w, h, Ub):
    nf = nf_of(cfg)
    out = np.empty((h, w, nf))
    lib().or_block_residual(C.byref(cfg), i0, j0, w, h, _a(Ub).reshape(-1), out.reshape(-1))
    return out


def tau(cfg: Cfg, Q):
    return lib().or_tau(C.byref(cfg), _a(Q))


def window_step(cfg: Cfg, U, i0, j0, w, h, dtv):
    """One step of the cells [i0,i0+w) x [j0,j0+h) of the full grid U (ny,nx,nf)
    computed on a margin-4 block cut out of U (periodic sides wrapped)."""
    ny, nx, nf = U.shape
    M = MARGIN
    My = 0 if ny == 1 else M
    per_x = cfg.side[0].base_type == BC_PERIODIC
    per_y = ny > 1 and cfg.side[2].base_type == BC_PERIODIC
    ii = np.arange(i0 - M, i0 + w + M)
    jj = np.arange(j0 - My, j0 + h + My)
    ii = np.mod(ii, nx) if per_x else np.clip(ii, 0, nx - 1)
    jj = np.mod(jj, ny) if per_y else np.clip(jj, 0, ny - 1)
    Ub = U[np.ix_(jj, ii)]
    return block_step(cfg, i0, j0, w, h, Ub, dtv)


# ---------------------------------------------------------------- tangent
_D2 = C.c_double * 2            # one dual number (value, derivative)


class SideT(C.Structure):
    _fields_ = [
        ("base_type", C.c_int),
        ("base_state", _D2 * 14),
        ("nspans", C.c_int),
        ("span_lo", C.c_double * MAX_SPANS),
        ("span_hi", C.c_double * MAX_SPANS),
        ("span_state", (_D2 * 14) * MAX_SPANS),
    ]


class CfgT(C.Structure):
    _fields_ = [
        ("system", C.c_int),
        ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("order", C.c_int), ("integrator", C.c_int), ("flux", C.c_int), ("limiter", C.c_int),
        ("cfl", C.c_double), ("sigma_lim", C.c_double), ("k_ws", C.c_double),
        ("tau_model", C.c_int),
        ("tau_ref", _D2), ("rho_ref", _D2), ("T_ref", _D2),
        ("side", SideT * 4),
        ("source_scheme", C.c_int),
        ("frozen_limiter", C.c_int),
    ]


_tlib = None


def tangent_lib():
    global _tlib
    if _tlib is None:
        L = C.CDLL(build_tangent())
        L.or_tangent_cfg_size.argtypes = []
        L.or_tangent_cfg_size.restype = C.c_size_t
        assert L.or_tangent_cfg_size() == C.sizeof(CfgT), "dual cfg layout mismatch"
        L.or_tangent_run.argtypes = [C.POINTER(CfgT), _dp, _dp, C.c_int, _dp, _dp, _dp]
        L.or_tangent_run.restype = C.c_int
        L.or_tangent_residual.argtypes = [C.POINTER(CfgT), _dp, _dp, _dp, _dp]
        L.or_tangent_residual.restype = C.c_int
        _tlib = L
    return _tlib


def tangent_cfg(cfg: Cfg, d_states=None, d_tau_ref=0.0, d_rho_ref=0.0, d_T_ref=0.0,
                frozen_limiter=False) -> CfgT:
    """Dual configuration: cfg's values with derivative directions for the
    imposed boundary states (d_states[s][0] = base state of side s,
    d_states[s][1 + n] = span n; primitive vectors of 14) and the
    relaxation parameters.  frozen_limiter: the shared limiter phi is held
    constant in the derivative (its value, hence the primal, unchanged)."""
    t = CfgT()
    t.frozen_limiter = 1 if frozen_limiter else 0
    for name in ("system", "nx", "ny", "x0", "x1", "y0", "y1", "order", "integrator", "flux",
                 "limiter", "cfl", "sigma_lim", "k_ws", "tau_model", "source_scheme"):
        setattr(t, name, getattr(cfg, name))
    for name, dv in (("tau_ref", d_tau_ref), ("rho_ref", d_rho_ref), ("T_ref", d_T_ref)):
        getattr(t, name)[0] = getattr(cfg, name)
        getattr(t, name)[1] = dv
    ds = np.zeros((4, 1 + MAX_SPANS, 14)) if d_states is None else np.asarray(d_states, float)
    for s in range(4):
        sd, st = cfg.side[s], t.side[s]
        st.base_type, st.nspans = sd.base_type, sd.nspans
        for k in range(14):
            st.base_state[k][0] = sd.base_state[k]
            st.base_state[k][1] = ds[s, 0, k]
        for n in range(MAX_SPANS):
            st.span_lo[n], st.span_hi[n] = sd.span_lo[n], sd.span_hi[n]
            for k in range(14):
                st.span_state[n][k][0] = sd.span_state[n][k]
                st.span_state[n][k][1] = ds[s, 1 + n, k]
    return t


def tangent_run(tcfg: CfgT, U, dU, dts):
    """n = len(dts) steps of the given sizes from U (ny, nx, nf) in the
    direction dU (and tcfg's directions).  Returns (U_n, dU_n)."""
    U = _a(U).reshape(tcfg.ny, tcfg.nx, -1)
    out, dout = np.empty_like(U), np.empty_like(U)
    dts = _a(dts)
    tangent_lib().or_tangent_run(C.byref(tcfg), U.reshape(-1), _a(dU).reshape(-1), len(dts),
                                 dts if len(dts) else np.zeros(1), out.reshape(-1),
                                 dout.reshape(-1))
    return out, dout


def tangent_residual(tcfg: CfgT, U, dU):
    """(L(U), dL) for non-periodic sides: the residual and its derivative."""
    U = _a(U).reshape(tcfg.ny, tcfg.nx, -1)
    L, dL = np.empty_like(U), np.empty_like(U)
    tangent_lib().or_tangent_residual(C.byref(tcfg), U.reshape(-1), _a(dU).reshape(-1),
                                      L.reshape(-1), dL.reshape(-1))
    return L, dL
