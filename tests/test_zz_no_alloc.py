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


def test_noalloc_matches_regular_entry_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as mx
    nx, Kn = 1000, 0.01
    prim = np.ascontiguousarray(wl.sod_prim(14, nx).T[:, None, :])
    ref = mx.Solver(system=14, nx=nx, ny=1)
    ref.set_state(prim)
    ref.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(Kn), 1.0, 1.0)
    U0 = ref.get_moments("conserved")                      # conserved initial state
    cfg = mx.make_config(system=14, nx=nx, ny=1)
    U = torch.from_numpy(U0.reshape(14, nx).copy()).cuda()
    t = 0.0
    for call in range(2):                                   # two calls in a row
        t_ref, n_ref = ref.step(60, 0.2)
        t, n = mx.mxe_tube_run_noalloc(cfg, U, t, 0.2, 60, tau_model=mx.TAU_HARDSPHERE,
                                       tau_ref=wl.sod_tau_ref(Kn))
        torch.cuda.synchronize()
        want = ref.get_moments("conserved").reshape(14, nx)
        got = U.cpu().numpy()
        err = np.linalg.norm(got - want, axis=1) / np.maximum(np.linalg.norm(want, axis=1), 1e-300)
        assert n == n_ref == 60
        assert t == pytest.approx(t_ref, rel=1e-12)
        assert err.max() <= 1e-12, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as mx
    cfg = mx.make_config(system=14, nx=16385, ny=1)
    U = torch.zeros((14, 16385), dtype=torch.float64, device="cuda")
    with pytest.raises(mx.MaxentError) as e:
        mx.mxe_tube_run_noalloc(cfg, U, 0.0, 1.0, 1)
    assert e.value.status == mx.EINVAL
