"""GB300-native solver for the fourth-order maximum-entropy moment method with
interpolative closure (Boccelli, Kaufmann, Magin & McDonald, JCP 2024).

This module is a thin ctypes binding of the C-ABI in ``include/maxent.h``
(library ``_lib/libmaxent.so``, CUDA for sm_103a).  It only marshals
arguments: every step of the method runs in the library's CUDA kernels.
The module-level functions carry the C names; ``Solver`` and ``Batch`` wrap
them for convenience.  Arrays are structure-of-arrays float64:
``(nf, ny, nx)`` for grids and the concatenation of ``(nf, ncells_b)`` for
batched tubes.  torch CUDA tensors are passed by device pointer.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

__all__ = [
    "Config", "Diag", "Solver", "Batch", "MaxentError", "lib",
    "mxe_create", "mxe_destroy", "mxe_set_stream", "mxe_get_stream", "mxe_set_state",
    "mxe_get_moments", "mxe_set_bc", "mxe_set_relaxation", "mxe_step", "mxe_step_dt",
    "mxe_get_diagnostics", "mxe_last_error", "mxe_batch_create", "mxe_batch_set_relaxation",
    "mxe_batch_get_clock", "mxe_batch_run", "mxe_set_mixed_policy", "mxe_tube_run_noalloc",
    "mxe_batch_autotune", "mxe_batch_set_shape", "mxe_set_dt_history", "mxe_get_dt_history",
    "mxe_adjoint_record", "mxe_adjoint_run", "mxe_adjoint_residual", "mxe_set_adjoint_precision",
    "mxe_set_stage_occupancy", "mxe_set_source_scheme", "mxe_set_adjoint_limiter",
    "mxe_set_face_packing", "mxe_batch_get_layout", "mxe_batch_plan_fill",
]

SOURCE_EXPLICIT, SOURCE_POINT_IMPLICIT = 0, 1
_SOURCE = {"explicit": SOURCE_EXPLICIT, "point_implicit": SOURCE_POINT_IMPLICIT}
OK, EINVAL, ENOMEM, ECUDA, EUNREALIZABLE, ENONFINITE, ETIMEOUT, ESTATE = range(8)
FP64, MIXED = 0, 1
FLUX_HLL, FLUX_RUSANOV = 0, 1
LIM_MINMOD, LIM_VANALBADA = 0, 1
FE, RK2 = 0, 1
BC_TRANSMISSIVE, BC_PERIODIC, BC_DIRICHLET = 0, 1, 2
XLO, XHI, YLO, YHI = 0, 1, 2, 3
TAU_NONE, TAU_CONST, TAU_HARDSPHERE = 0, 1, 2
PRIMITIVE, CONSERVED, SIGMA, CONSERVED_RESTORE = 0, 1, 2, 3
_KINDS = {"primitive": PRIMITIVE, "conserved": CONSERVED, "sigma": SIGMA,
          "restore": CONSERVED_RESTORE}


class Config(C.Structure):
    _fields_ = [
        ("system", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("precision", C.c_int), ("flux", C.c_int), ("limiter", C.c_int),
        ("order", C.c_int), ("integrator", C.c_int),
        ("cfl", C.c_double), ("sigma_lim", C.c_double), ("k_ws", C.c_double),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("last_dt", C.c_double), ("steps", C.c_longlong),
        ("max_rate", C.c_double), ("min_sigma", C.c_double),
        ("n_sigma_below_lim", C.c_longlong), ("n_sigma_above_one", C.c_longlong),
        ("n_nonpositive", C.c_longlong), ("n_nonfinite", C.c_longlong),
        ("n_fp64_closures", C.c_longlong), ("n_closures", C.c_longlong),
        ("sums", C.c_double * 14),
        ("planar", C.c_longlong),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "sums"}
        d["sums"] = list(self.sums)
        return d


class MaxentError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"maxent status {status}: {msg}")
        self.status = status


_lib = None
_P = C.c_void_p


def lib():
    """Load libmaxent.so (building it first if sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        sig = {
            "mxe_create": ([C.POINTER(Config), C.POINTER(_P)], C.c_int),
            "mxe_destroy": ([_P], None),
            "mxe_set_stream": ([_P, _P], C.c_int),
            "mxe_get_stream": ([_P], _P),
            "mxe_set_state": ([_P, C.c_int, _P, C.c_int], C.c_int),
            "mxe_get_moments": ([_P, C.c_int, _P, C.c_int], C.c_int),
            "mxe_set_bc": ([_P, C.c_int, C.c_int, C.c_double, C.c_double, _P], C.c_int),
            "mxe_set_relaxation": ([_P, C.c_int, C.c_double, C.c_double, C.c_double], C.c_int),
            "mxe_step": ([_P, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int)],
                         C.c_int),
            "mxe_step_dt": ([_P, C.c_int, _P], C.c_int),
            "mxe_get_diagnostics": ([_P, C.POINTER(Diag)], C.c_int),
            "mxe_last_error": ([_P], C.c_char_p),
            "mxe_batch_create": ([C.POINTER(Config), C.c_int, _P, _P, C.POINTER(_P)], C.c_int),
            "mxe_batch_set_relaxation": ([_P, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double], C.c_int),
            "mxe_batch_get_clock": ([_P, _P, _P], C.c_int),
            "mxe_batch_run": ([_P, C.c_int, C.c_double], C.c_int),
            "mxe_batch_autotune": ([_P, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)], C.c_int),
            "mxe_batch_set_shape": ([_P, C.c_int, C.c_int], C.c_int),
            "mxe_batch_get_layout": ([_P, _P, _P, _P], C.c_int),
            "mxe_batch_plan_fill": ([C.c_int, _P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                                     _P], C.c_int),
            "mxe_set_dt_history": ([_P, C.c_longlong], C.c_int),
            "mxe_get_dt_history": ([_P, C.c_longlong, _P], C.c_int),
            "mxe_adjoint_record": ([_P, C.c_int, _P], C.c_int),
            "mxe_set_adjoint_precision": ([_P, C.c_int], C.c_int),
            "mxe_adjoint_run": ([_P, _P, C.c_int, _P, _P], C.c_int),
            "mxe_adjoint_residual": ([_P, _P, _P, _P, C.c_int, _P, _P], C.c_int),
            "mxe_set_mixed_policy": ([_P, C.c_double, C.c_double, C.c_double, C.c_int], C.c_int),
            "mxe_set_stage_occupancy": ([_P, C.c_int], C.c_int),
            "mxe_set_face_packing": ([_P, C.c_int], C.c_int),
            "mxe_set_source_scheme": ([_P, C.c_int], C.c_int),
            "mxe_set_adjoint_limiter": ([_P, C.c_int], C.c_int),
            "mxe_tube_run_noalloc": ([C.POINTER(Config), C.c_int, C.c_int, C.c_int, C.c_double,
                                      C.c_double, C.c_double, _P, C.c_double, C.c_double,
                                      C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int), _P],
                                     C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(ctx, st):
    if st != OK:
        msg = lib().mxe_last_error(ctx).decode() if ctx else ""
        raise MaxentError(st, msg)


# Elements per field of every live context (cells of a grid, or of all tubes
# of a batch), so that every wrapper can check the size of the arrays it
# hands to the library: the library trusts its pointers.
_CELLS = {}
_NF = {}


def _ctx_key(ctx):
    return ctx.value if hasattr(ctx, "value") else int(ctx)


def _ptr(a, nelem=None):
    """(pointer, on_device) of a numpy array or a CUDA tensor (float64,
    contiguous).  nelem: required number of elements.  A CUDA tensor must
    live on the current device, where the library launches its kernels."""
    if hasattr(a, "data_ptr"):
        if a.dtype.__repr__() != "torch.float64" or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        if a.is_cuda:
            import torch
            if a.device.index != torch.cuda.current_device():
                raise ValueError(f"tensor on {a.device}, but the current device is "
                                 f"cuda:{torch.cuda.current_device()}")
        if nelem is not None and a.numel() != nelem:
            raise ValueError(f"tensor holds {a.numel()} elements, {nelem} expected")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous float64")
    if nelem is not None and a.size != nelem:
        raise ValueError(f"array holds {a.size} elements, {nelem} expected")
    return C.c_void_p(a.ctypes.data), 0


def _state_elems(ctx, kind=None):
    """Elements of a state array of this context (one field for SIGMA)."""
    k = _ctx_key(ctx)
    if k not in _CELLS:
        raise ValueError("unknown or destroyed context")
    return _CELLS[k] * (1 if kind == SIGMA else _NF[k])


# ------------------------------------------------------------ C-named wrappers
def mxe_create(cfg: Config):
    h = _P()
    st = lib().mxe_create(C.byref(cfg), C.byref(h))
    if st != OK:
        raise MaxentError(st, "mxe_create rejected the configuration")
    _CELLS[_ctx_key(h)] = int(cfg.nx) * int(cfg.ny)
    _NF[_ctx_key(h)] = int(cfg.system)
    return h


def mxe_destroy(ctx):
    _CELLS.pop(_ctx_key(ctx), None)
    _NF.pop(_ctx_key(ctx), None)
    lib().mxe_destroy(ctx)


def mxe_set_stream(ctx, stream_ptr):
    _check(ctx, lib().mxe_set_stream(ctx, _P(stream_ptr)))


def mxe_get_stream(ctx):
    return lib().mxe_get_stream(ctx)


def mxe_set_state(ctx, kind, arr):
    p, dev = _ptr(arr, _state_elems(ctx, kind))
    _check(ctx, lib().mxe_set_state(ctx, kind, p, dev))


def mxe_get_moments(ctx, kind, out):
    p, dev = _ptr(out, _state_elems(ctx, kind))
    _check(ctx, lib().mxe_get_moments(ctx, kind, p, dev))
    return out


def mxe_set_bc(ctx, side, bctype, lo=0.0, hi=0.0, prim=None):
    buf = None
    if prim is not None:
        buf = np.ascontiguousarray(np.asarray(prim, dtype=np.float64))
    _check(ctx, lib().mxe_set_bc(ctx, side, bctype, lo, hi,
                                 _P(buf.ctypes.data) if buf is not None else None))


def mxe_set_relaxation(ctx, model, tau_ref=1.0, rho_ref=1.0, T_ref=1.0):
    _check(ctx, lib().mxe_set_relaxation(ctx, model, tau_ref, rho_ref, T_ref))


def mxe_step(ctx, max_steps, t_end, sync=True):
    if not sync:
        _check(ctx, lib().mxe_step(ctx, max_steps, t_end, None, None))
        return None
    t = C.c_double()
    n = C.c_int()
    _check(ctx, lib().mxe_step(ctx, max_steps, t_end, C.byref(t), C.byref(n)))
    return t.value, n.value


def mxe_step_dt(ctx, dts):
    d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    _check(ctx, lib().mxe_step_dt(ctx, d.size, _P(d.ctypes.data)))


def mxe_get_diagnostics(ctx):
    d = Diag()
    _check(ctx, lib().mxe_get_diagnostics(ctx, C.byref(d)))
    return d.as_dict()


def mxe_last_error(ctx):
    return lib().mxe_last_error(ctx).decode()


def mxe_set_mixed_policy(ctx, sigma_lo=0.0, sigma_hi=0.999, det_min=1e-3, resync_every=16):
    _check(ctx, lib().mxe_set_mixed_policy(ctx, sigma_lo, sigma_hi, det_min, resync_every))


def mxe_set_adjoint_limiter(ctx, frozen):
    _check(ctx, lib().mxe_set_adjoint_limiter(ctx, 1 if frozen else 0))


def mxe_set_source_scheme(ctx, scheme):
    _check(ctx, lib().mxe_set_source_scheme(ctx, scheme))


def mxe_set_stage_occupancy(ctx, blocks_per_sm):
    _check(ctx, lib().mxe_set_stage_occupancy(ctx, blocks_per_sm))


def mxe_set_face_packing(ctx, packed):
    _check(ctx, lib().mxe_set_face_packing(ctx, int(packed)))


def mxe_tube_run_noalloc(cfg: Config, U_dev, t0, t_end, max_steps, bc_lo=BC_TRANSMISSIVE,
                         bc_hi=BC_TRANSMISSIVE, tau_model=TAU_NONE, tau_ref=1.0, rho_ref=1.0,
                         T_ref=1.0, stream=None):
    """1D solve on a caller-owned device array (torch CUDA float64 tensor,
    conserved SoA (nf, nx)) using only the library's fixed device arrays.
    U must hold exactly nf*nx elements and live on the current device."""
    p, dev = _ptr(U_dev, int(cfg.system) * int(cfg.nx))
    if not dev:
        raise ValueError("U must be a device tensor")
    t = C.c_double()
    n = C.c_int()
    st = lib().mxe_tube_run_noalloc(C.byref(cfg), bc_lo, bc_hi, tau_model, tau_ref, rho_ref,
                                    T_ref, p, t0, t_end, max_steps, C.byref(t), C.byref(n),
                                    _P(stream) if stream else None)
    if st != OK:
        raise MaxentError(st, "mxe_tube_run_noalloc failed")
    return t.value, n.value


def mxe_batch_create(cfg: Config, ncells, lengths):
    nc = np.ascontiguousarray(np.asarray(ncells, dtype=np.int32))
    ln = np.ascontiguousarray(np.asarray(lengths, dtype=np.float64))
    h = _P()
    st = lib().mxe_batch_create(C.byref(cfg), nc.size, _P(nc.ctypes.data), _P(ln.ctypes.data),
                                C.byref(h))
    if st != OK:
        raise MaxentError(st, "mxe_batch_create rejected the configuration")
    _CELLS[_ctx_key(h)] = int(nc.sum())
    _NF[_ctx_key(h)] = int(cfg.system)
    return h


def mxe_batch_set_relaxation(ctx, tube, model, tau_ref=1.0, rho_ref=1.0, T_ref=1.0):
    _check(ctx, lib().mxe_batch_set_relaxation(ctx, tube, model, tau_ref, rho_ref, T_ref))


def mxe_batch_get_clock(ctx, n):
    t = np.zeros(n)
    s = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().mxe_batch_get_clock(ctx, _P(t.ctypes.data), _P(s.ctypes.data)))
    return t, s


def mxe_batch_run(ctx, max_steps, t_end):
    _check(ctx, lib().mxe_batch_run(ctx, max_steps, t_end))


GHOST_SLOTS = 5                  # base Dirichlet state + 4 spans per side


def mxe_set_dt_history(ctx, capacity):
    _check(ctx, lib().mxe_set_dt_history(ctx, int(capacity)))


def mxe_get_dt_history(ctx, n):
    out = np.empty(int(n))
    _check(ctx, lib().mxe_get_dt_history(ctx, int(n), C.c_void_p(out.ctypes.data)))
    return out


def mxe_set_adjoint_precision(ctx, precision):
    _check(ctx, lib().mxe_set_adjoint_precision(ctx, _ENUM[precision] if isinstance(precision, str)
                                                else int(precision)))


def mxe_adjoint_record(ctx, dts, n=None):
    """dts: step sizes to replay, or None to record n CFL steps."""
    if dts is None:
        _check(ctx, lib().mxe_adjoint_record(ctx, int(n), None))
        return
    d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    _check(ctx, lib().mxe_adjoint_record(ctx, len(d), C.c_void_p(d.ctypes.data)))


def mxe_adjoint_run(ctx, ubar):
    """ubar: adjoint of the final state (numpy or CUDA tensor, (14, ny, nx)),
    overwritten with the adjoint of the first recorded state.  Returns
    (gbar [4, GHOST_SLOTS, 14], taubar)."""
    p, dev = _ptr(ubar, _state_elems(ctx))
    gb = np.zeros((4, GHOST_SLOTS, 14))
    tb = C.c_double(0.0)
    _check(ctx, lib().mxe_adjoint_run(ctx, p, dev, C.c_void_p(gb.ctypes.data), C.byref(tb)))
    return gb, tb.value


def mxe_adjoint_residual(ctx, U, V, out):
    n = _state_elems(ctx)
    pu, du = _ptr(U, n)
    pv, dv = _ptr(V, n)
    po, do = _ptr(out, n)
    if not (du == dv == do):
        raise ValueError("U, V and out must all be on the host or all on the device")
    gb = np.zeros((4, GHOST_SLOTS, 14))
    tb = C.c_double(0.0)
    _check(ctx, lib().mxe_adjoint_residual(ctx, pu, pv, po, du, C.c_void_p(gb.ctypes.data),
                                           C.byref(tb)))
    return out, gb, tb.value


def mxe_batch_autotune(ctx, t_probe):
    nt, cl, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
    _check(ctx, lib().mxe_batch_autotune(ctx, t_probe, C.byref(nt), C.byref(cl), C.byref(ms)))
    return nt.value, cl.value, ms.value


def mxe_batch_set_shape(ctx, nt, cl):
    _check(ctx, lib().mxe_batch_set_shape(ctx, nt, cl))


def mxe_batch_plan_fill(cells, steps, chunk, cl, teams, fill):
    """Host-only: (tubes for the teams, estimated time) for tubes in work order."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    steps = np.ascontiguousarray(steps, dtype=np.float64)
    if cells.shape != steps.shape or cells.ndim != 1:
        raise ValueError("cells and steps must be 1-D arrays of the same length")
    nA, t = C.c_int(), C.c_double()
    st = lib().mxe_batch_plan_fill(len(cells), cells.ctypes.data, steps.ctypes.data, chunk, cl,
                                   teams, fill, C.byref(nA), C.byref(t))
    if st != OK:
        raise MaxentError(st, "mxe_batch_plan_fill: invalid arguments")
    return nA.value, t.value


def mxe_batch_get_layout(ctx):
    teams, tubes, fill = C.c_int(), C.c_int(), C.c_int()
    _check(ctx, lib().mxe_batch_get_layout(ctx, C.byref(teams), C.byref(tubes), C.byref(fill)))
    return teams.value, tubes.value, fill.value


# ------------------------------------------------------------ convenience
_ENUM = {
    "fp64": FP64, "mixed": MIXED, "hll": FLUX_HLL, "rusanov": FLUX_RUSANOV,
    "minmod": LIM_MINMOD, "vanalbada": LIM_VANALBADA, "fe": FE, "rk2": RK2,
}


def make_config(system=14, nx=64, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, precision="fp64",
                flux="hll", limiter="minmod", order=2, integrator="rk2", cfl=0.5,
                sigma_lim=1e-4, k_ws=1.0) -> Config:
    e = lambda v: _ENUM[v] if isinstance(v, str) else int(v)
    return Config(system, nx, ny, x0, x1, y0, y1, e(precision), e(flux), e(limiter), order,
                  e(integrator), cfl, sigma_lim, k_ws)


class Solver:
    """One grid (ny == 1: a single 1D problem)."""

    def __init__(self, **kw):
        self.cfg = make_config(**kw)
        self.nf = self.cfg.system
        self.ctx = mxe_create(self.cfg)
        self.shape = (self.nf, self.cfg.ny, self.cfg.nx)

    def close(self):
        if getattr(self, "ctx", None):
            mxe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        mxe_set_stream(self.ctx, stream_ptr)

    @property
    def stream(self):
        return mxe_get_stream(self.ctx)

    def set_state(self, arr, kind="primitive"):
        if isinstance(arr, np.ndarray):
            arr = np.ascontiguousarray(arr, dtype=np.float64)
        mxe_set_state(self.ctx, _KINDS[kind], arr)

    def get_moments(self, kind="primitive", out=None):
        if out is None:
            shape = (1,) + self.shape[1:] if kind == "sigma" else self.shape
            out = np.empty(shape)
        return mxe_get_moments(self.ctx, _KINDS[kind], out)

    def set_bc(self, side, bctype, lo=0.0, hi=0.0, state=None):
        mxe_set_bc(self.ctx, side, bctype, lo, hi, state)

    def set_relaxation(self, model, tau_ref=1.0, rho_ref=1.0, T_ref=1.0):
        mxe_set_relaxation(self.ctx, model, tau_ref, rho_ref, T_ref)

    def step(self, max_steps, t_end=float("inf"), sync=True):
        return mxe_step(self.ctx, max_steps, t_end, sync)

    def step_dt(self, dts):
        mxe_step_dt(self.ctx, dts)

    def diagnostics(self):
        return mxe_get_diagnostics(self.ctx)

    def set_dt_history(self, capacity):
        mxe_set_dt_history(self.ctx, capacity)

    def dt_history(self, n):
        return mxe_get_dt_history(self.ctx, n)

    def set_adjoint_precision(self, precision):
        mxe_set_adjoint_precision(self.ctx, precision)

    def adjoint_record(self, dts, n=None):
        """Replay the given step sizes keeping the tape, or (dts None)
        march n CFL steps keeping the tape (needs the dt history)."""
        mxe_adjoint_record(self.ctx, dts, n)

    def adjoint_run(self, ubar):
        return mxe_adjoint_run(self.ctx, ubar)

    def adjoint_residual(self, U, V, out=None):
        if out is None:
            out = np.empty(self.shape)
        return mxe_adjoint_residual(self.ctx, U, V, out)

    def set_mixed_policy(self, sigma_lo=0.0, sigma_hi=0.999, det_min=1e-3, resync_every=16):
        mxe_set_mixed_policy(self.ctx, sigma_lo, sigma_hi, det_min, resync_every)

    def set_adjoint_limiter(self, frozen):
        """False: exact derivative of the limiter branch; True: phi held
        constant in the adjoint."""
        mxe_set_adjoint_limiter(self.ctx, frozen)

    def set_source_scheme(self, scheme):
        """"explicit" (BGK source in the stage residual) or "point_implicit"
        (backward-Euler relaxation after each stage)."""
        mxe_set_source_scheme(self.ctx, _SOURCE[scheme] if isinstance(scheme, str) else scheme)

    def set_stage_occupancy(self, blocks_per_sm):
        """Planar mixed stage kernel: 3 (default) or 2 blocks per SM."""
        mxe_set_stage_occupancy(self.ctx, blocks_per_sm)

    def set_face_packing(self, packed):
        """Planar mixed stage at 3 blocks per SM: True (default) evaluates
        the two face states of a face as one packed FP32 pair."""
        mxe_set_face_packing(self.ctx, packed)


class Batch(Solver):
    """Independent 1D tubes advanced in one persistent launch."""

    def __init__(self, ncells, lengths, **kw):
        if len(ncells) == 0 or len(ncells) != len(lengths):
            raise MaxentError(EINVAL, "need one length per tube and at least one tube")
        kw.setdefault("ny", 1)
        kw["nx"] = int(max(ncells))
        self.cfg = make_config(**kw)
        self.nf = self.cfg.system
        self.ncells = [int(n) for n in ncells]
        self.ctx = mxe_batch_create(self.cfg, self.ncells, lengths)
        self.shape = (self.nf * sum(self.ncells),)

    def pack(self, tubes):
        """list of (nf, n_b) arrays -> concatenated SoA"""
        return np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).ravel()
                                                    for t in tubes]))

    def unpack(self, flat, nf=None):
        nf = nf or self.nf
        out, o = [], 0
        for n in self.ncells:
            out.append(flat[o:o + nf * n].reshape(nf, n))
            o += nf * n
        return out

    def get_moments(self, kind="primitive", out=None):
        if out is None:
            out = np.empty(sum(self.ncells) if kind == "sigma" else self.shape)
        return mxe_get_moments(self.ctx, _KINDS[kind], out)

    def set_tube_relaxation(self, tube, model, tau_ref=1.0, rho_ref=1.0, T_ref=1.0):
        mxe_batch_set_relaxation(self.ctx, tube, model, tau_ref, rho_ref, T_ref)

    def clock(self):
        return mxe_batch_get_clock(self.ctx, len(self.ncells))

    def run(self, max_steps, t_end):
        mxe_batch_run(self.ctx, max_steps, t_end)

    def autotune(self, t_probe):
        """Time every block shape over t_probe (state restored); returns
        (threads per CTA, CTAs per team, ms of the fastest)."""
        return mxe_batch_autotune(self.ctx, t_probe)

    def set_shape(self, nt, cl):
        mxe_batch_set_shape(self.ctx, nt, cl)

    def layout(self):
        """(teams, tubes handed to the teams, CTAs of the fill launch)."""
        return mxe_batch_get_layout(self.ctx)
