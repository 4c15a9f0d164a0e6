"""The OpenMP timing build of the oracle (the CPU baseline's all-core leg)
must compute exactly what the serial oracle computes: same arithmetic per
cell, same order of contributions, only the rows and columns shared among
threads.  CPU only."""
import os

import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import jets_oracle_cfg


@pytest.fixture(scope="module")
def omp4():
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    import oracle
    oracle.build(omp=True)
    return oracle


def test_omp_build_uses_several_threads(omp4):
    assert omp4.threads(omp=False) == 1
    assert omp4.threads(omp=True) >= 2


@pytest.mark.parametrize("integ", [0, 1])
def test_omp_step_bitwise_equal_2d_jets(omp4, integ):
    orc = omp4
    n = 24
    setup = wl.jets_setup(Kn=0.1)
    prim = wl.jets_like_field(n, n + 3, setup)          # (ny, nx, 14), nx != ny
    U = orc.prim2cons_field(prim)
    cfg = jets_oracle_cfg(orc, n + 3, n, setup, integ=integ)
    d1 = orc.dt(cfg, U, 0.0, 10.0)
    d2 = orc.dt(cfg, U, 0.0, 10.0, omp=True)
    assert d1 == d2
    A = orc.step(cfg, U, d1)
    B = orc.step(cfg, U, d1, omp=True)
    assert np.array_equal(A, B)


@pytest.mark.parametrize("system", [5, 14])
def test_omp_run_bitwise_equal_sod(omp4, system):
    orc = omp4
    nx = 200
    prim = wl.sod_prim(system, nx)[None]
    U = orc.prim2cons_field(prim)
    cfg = orc.make_cfg(system=system, nx=nx, ny=1, order=1 if system == 5 else 2,
                       integrator=orc.FE if system == 5 else orc.RK2,
                       tau_model=orc.TAU_HARDSPHERE, tau_ref=wl.sod_tau_ref(0.01))
    A, ta, ha = orc.run(cfg, U, 0.0, 0.2, 40)
    B, tb, hb = orc.run(cfg, U, 0.0, 0.2, 40, omp=True)
    assert ta == tb and np.array_equal(ha, hb) and np.array_equal(A, B)
