"""Shared helpers of the test-suite (layout conversion, error norms, builders).

Inputs always come from ``paper_2401_15233_gb300.workloads`` (seeded
generators); expected values always come from the oracle.
"""
from __future__ import annotations

import numpy as np

from paper_2401_15233_gb300 import workloads as wl


def aos_to_soa(U):
    """(ny, nx, nf) -> (nf, ny, nx)"""
    return np.ascontiguousarray(np.moveaxis(U, -1, 0))


def soa_to_aos(U):
    return np.ascontiguousarray(np.moveaxis(U, 0, -1))


def cons_field(orc, prim):
    """primitive (..., nf) -> conserved via the oracle, cell by cell"""
    return orc.prim2cons_field(prim)


def prim_field(orc, U):
    return orc.cons2prim_field(U)


def field_rel_err(a, b, axis_field=-1):
    """Normwise relative error per field: ||a_k - b_k||_2 / ||b_k||_2.
    Fields that are identically zero in b are measured against the largest
    field norm of b (they must stay (near) zero)."""
    a = np.moveaxis(np.asarray(a), axis_field, 0).reshape(a.shape[axis_field], -1)
    b = np.moveaxis(np.asarray(b), axis_field, 0).reshape(b.shape[axis_field], -1)
    nb = np.linalg.norm(b, axis=1)
    ref = np.where(nb > 0, nb, nb.max())
    return np.linalg.norm(a - b, axis=1) / ref


def jets_oracle_cfg(orc, nx, ny, setup, order=2, integ=1, flux=0, limiter=0, cfl=0.5,
                    sigma_lim=1e-4):
    lo, hi = setup["slot"]
    sides = [
        {"type": 0, "spans": [(lo, hi, setup["left"])]},
        {"type": 0},
        {"type": 0, "spans": [(lo, hi, setup["bottom"])]},
        {"type": 0},
    ]
    return orc.make_cfg(system=14, nx=nx, ny=ny, order=order, integrator=integ, flux=flux,
                        limiter=limiter, cfl=cfl, sigma_lim=sigma_lim, tau_model=2,
                        tau_ref=setup["tau_ref"], rho_ref=setup["rho_ref"],
                        T_ref=setup["T_ref"], sides=sides)


def jets_gpu_solver(mx, nx, ny, setup, precision="fp64", order=2, integrator="rk2",
                    flux="hll", limiter="minmod", cfl=0.5, sigma_lim=1e-4):
    s = mx.Solver(system=14, nx=nx, ny=ny, precision=precision, order=order,
                  integrator=integrator, flux=flux, limiter=limiter, cfl=cfl,
                  sigma_lim=sigma_lim)
    lo, hi = setup["slot"]
    s.set_bc(mx.XLO, mx.BC_DIRICHLET, lo, hi, setup["left"])
    s.set_bc(mx.YLO, mx.BC_DIRICHLET, lo, hi, setup["bottom"])
    s.set_relaxation(mx.TAU_HARDSPHERE, setup["tau_ref"], setup["rho_ref"], setup["T_ref"])
    return s
