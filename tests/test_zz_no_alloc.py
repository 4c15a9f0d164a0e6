"""The fixed-scratch 1D entry point (mxe_tube_run_noalloc) against the regular
entry point.  It exists for callers that cannot allocate device memory (a
host whose device memory is owned by its own pool allocator, or a loop that
cannot afford cudaMalloc's device synchronisation); it must give the same
result as mxe_step on the same problem, call after call, although every call
reuses the same fixed device arrays.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAX_CELLS = 16384            # the entry point's fixed stage buffer holds 14 x 16384 doubles


def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("system", [5, 14])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
@pytest.mark.parametrize("nx", [1000, MAX_CELLS])
def test_noalloc_matches_regular_entry_two_calls_in_a_row(system, bc, nx):
    torch = _need_cuda()
    import paper_2401_15233_gb300 as mx
    Kn = 0.01
    steps = 40 if nx <= 1000 else 6          # the largest size fills the whole fixed stage buffer
    bct = mx.BC_PERIODIC if bc == "periodic" else mx.BC_TRANSMISSIVE
    prim = np.ascontiguousarray(wl.sod_prim(system, nx).T[:, None, :])
    ref = mx.Solver(system=system, nx=nx, ny=1)
    if bct == mx.BC_PERIODIC:
        ref.set_bc(mx.XLO, mx.BC_PERIODIC)
        ref.set_bc(mx.XHI, mx.BC_PERIODIC)
    ref.set_state(prim)
    ref.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(Kn), 1.0, 1.0)
    U0 = ref.get_moments("conserved")                      # conserved initial state
    cfg = mx.make_config(system=system, nx=nx, ny=1)
    U = torch.from_numpy(U0.reshape(system, nx).copy()).cuda()
    t = 0.0
    for call in range(2):                                   # two calls in a row
        t_ref, n_ref = ref.step(steps, 0.2)
        t, n = mx.mxe_tube_run_noalloc(cfg, U, t, 0.2, steps, bc_lo=bct, bc_hi=bct,
                                       tau_model=mx.TAU_HARDSPHERE, tau_ref=wl.sod_tau_ref(Kn))
        torch.cuda.synchronize()
        want = ref.get_moments("conserved").reshape(system, nx)
        got = U.cpu().numpy()
        err = np.linalg.norm(got - want, axis=1) / np.maximum(np.linalg.norm(want, axis=1), 1e-300)
        assert n == n_ref == steps
        assert t == pytest.approx(t_ref, rel=1e-12)
        assert err.max() <= 1e-12, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = _need_cuda()
    import paper_2401_15233_gb300 as mx
    cfg = mx.make_config(system=14, nx=MAX_CELLS + 1, ny=1)
    U = torch.zeros((14, MAX_CELLS + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(mx.MaxentError) as e:
        mx.mxe_tube_run_noalloc(cfg, U, 0.0, 1.0, 1)
    assert e.value.status == mx.EINVAL


def test_noalloc_binding_rejects_a_short_array():
    """The library cannot see a raw pointer's extent; the binding refuses a
    tensor that does not hold nf*nx elements before anything is launched."""
    torch = _need_cuda()
    import paper_2401_15233_gb300 as mx
    cfg = mx.make_config(system=14, nx=1000, ny=1)
    U = torch.zeros((14, 999), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        mx.mxe_tube_run_noalloc(cfg, U, 0.0, 1.0, 1)
