"""Batched 14-moment Sod tubes in mixed precision (one persistent launch,
teams of CTAs, work queue, CUDA graph replay, autotuned block shape).

Bounds (stated before measuring), as for the 2D mixed path: one mixed step
from the oracle's state within 1e-4 normwise per field (FP32 arithmetic
sanity bound); a free run's per-field L1 error within 10x the L1 difference
between two FP64 oracle runs whose initial data differ by a 1e-7 relative
perturbation.  The block shape and the work order change only which CTA
computes a cell, never the arithmetic: results are bitwise identical."""
import numpy as np
import pytest

from paper_2401_15233_gb300 import workloads as wl
from tests._util import aos_to_soa, cons_field, field_rel_err, soa_to_aos

pytestmark = pytest.mark.gpu

SHAPES = [(128, 1), (256, 1), (128, 2), (256, 4), (128, 8)]


@pytest.fixture(scope="module")
def mx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_15233_gb300 as m
    m.lib()
    return m


def l1_rel(a, b):
    a = a.reshape(-1, a.shape[-1]); b = b.reshape(-1, b.shape[-1])
    den = np.abs(b).sum(0)
    return np.abs(a - b).sum(0) / np.where(den > 0, den, 1.0)


def sod_batch(mx, tubes, shape=None):
    b = mx.Batch([t[0] for t in tubes], [1.0] * len(tubes), system=14, precision="mixed")
    b.set_state(b.pack([aos_to_soa(wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None])[:, 0]
                        for (nc, kn, r) in tubes]))
    for i, (nc, kn, r) in enumerate(tubes):
        b.set_tube_relaxation(i, mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
    if shape:
        b.set_shape(*shape)
    return b


def oracle_cfg(orc, nc, kn):
    return orc.make_cfg(system=14, nx=nc, ny=1, tau_model=2, tau_ref=wl.sod_tau_ref(kn))


def step_sensitivity(orc, cfg, U, dt, rng):
    """Per-field normwise change of one FP64 oracle step when every primitive
    of the input is perturbed by 1e-7 relative (the data resolution of FP32)."""
    prim = orc.cons2prim_field(U)
    Up = orc.prim2cons_field(prim * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=prim.shape)))
    return field_rel_err(orc.step(cfg, Up, dt), orc.step(cfg, U, dt))


def test_mixed_tubes_per_step(mx, orc):
    """One mixed step per launch from the oracle's state, every tube on its own
    clock and Knudsen number.  Bound per field: 1e-4 (the 2D sanity bound), or
    10x the oracle step's own sensitivity to a 1e-7 data perturbation where
    that is larger -- early Sod steps are such a case: the shared limiter
    divides increments that are small against the state itself."""
    tubes = wl.batch_tubes(6, nmin=40, nmax=300)
    b = sod_batch(mx, tubes)
    Us = [cons_field(orc, wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None]) for (nc, kn, r) in tubes]
    cfgs = [oracle_cfg(orc, nc, kn) for (nc, kn, r) in tubes]
    rng = np.random.default_rng(3)
    worst = 0.0
    for step in range(10):
        b.set_state(b.pack([aos_to_soa(U)[:, 0] for U in Us]), kind="conserved")
        b.run(1, 0.2)
        out = b.unpack(b.get_moments("conserved"))
        for i in range(len(tubes)):
            dt = orc.dt(cfgs[i], Us[i], 0.0, 0.2)
            sens = step_sensitivity(orc, cfgs[i], Us[i], dt, rng)
            Us[i] = orc.step(cfgs[i], Us[i], dt)
            err = field_rel_err(soa_to_aos(out[i][:, None, :]), Us[i])
            assert (err <= np.maximum(1e-4, 10 * sens)).all(), (step, i, err, sens)
            worst = max(worst, err.max())
    d = b.diagnostics()
    assert d["planar"] == 1 and d["n_closures"] > 0
    print(f"mixed tubes per-step error max {worst:.2e}; FP64 closures "
          f"{d['n_fp64_closures']} of {d['n_closures']}")


def test_mixed_tubes_shape_invariance(mx):
    """Every block shape (threads x team size) gives bitwise the same batch."""
    tubes = wl.batch_tubes(12, nmin=100, nmax=1500)
    ref = None
    for shape in SHAPES:
        b = sod_batch(mx, tubes, shape)
        b.run(10 ** 6, 0.01)
        U = b.get_moments("conserved")
        t, st = b.clock()
        assert np.allclose(t, 0.01, rtol=0, atol=1e-15)
        if ref is None:
            ref = (U, st)
        else:
            assert np.array_equal(U, ref[0]), shape
            assert np.array_equal(st, ref[1]), shape


def test_mixed_tubes_fill_launch(mx):
    """More tubes than 8-CTA teams: the team launch leaves CTA slots unused
    (clusters are placed whole), and a concurrent launch of single CTAs takes
    the smallest tubes (the division uses each tube's step estimate from
    its current CFL rate).  The layout of the run shows both launches; the
    batch is bitwise the single-CTA (128 x 1) batch, also after a graph
    re-capture for a new t_end."""
    tubes = wl.batch_tubes(64, nmin=100, nmax=3000)
    b = sod_batch(mx, tubes, (256, 8))
    b.run(10 ** 6, 0.01)
    teams, team_tubes, fill = b.layout()
    print(f"layout 256 x 8: {teams} teams take {team_tubes} tubes, {fill} fill CTAs "
          f"take {len(tubes) - team_tubes}")
    assert fill > 0 and 0 < team_tubes < len(tubes) and teams <= team_tubes
    ref = sod_batch(mx, tubes, (128, 1))
    assert ref.layout()[2] == 0
    ref.run(10 ** 6, 0.01)
    assert np.array_equal(b.get_moments("conserved"), ref.get_moments("conserved"))
    t, st = b.clock()
    tr, sr = ref.clock()
    assert np.array_equal(st, sr) and np.allclose(t, 0.01, rtol=0, atol=1e-15)
    b.run(10 ** 6, 0.02)                   # a new t_end: re-captured graph with both launches
    ref.run(10 ** 6, 0.02)
    assert np.array_equal(b.get_moments("conserved"), ref.get_moments("conserved"))


def test_mixed_batch_equals_single_tubes(mx):
    """The work queue hands tubes out in any order: each tube of the batch is
    bitwise the tube run alone in its own context."""
    tubes = wl.batch_tubes(5, nmin=60, nmax=700)
    b = sod_batch(mx, tubes, (128, 2))
    b.run(10 ** 6, 0.02)
    outs = b.unpack(b.get_moments("conserved"))
    for i, (nc, kn, r) in enumerate(tubes):
        s = mx.Solver(system=14, nx=nc, ny=1, precision="mixed")
        s.set_state(aos_to_soa(wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None])[:, 0])
        s.set_relaxation(mx.TAU_HARDSPHERE, wl.sod_tau_ref(kn), 1.0, 1.0)
        s.step(10 ** 6, 0.02)
        assert np.array_equal(s.get_moments("conserved").reshape(14, nc), outs[i]), i


def test_mixed_tubes_graph_replay(mx):
    """Repeated runs replay the captured graph; a run after t_end is a no-op;
    a new t_end re-captures; a changed relaxation time re-captures too."""
    tubes = wl.batch_tubes(4, nmin=80, nmax=400)
    b = sod_batch(mx, tubes)
    for _ in range(3):
        b.run(5, 0.03)                     # same arguments: graph replay
    t, st = b.clock()
    assert (st == 15).all(), st
    b.run(10 ** 6, 0.03)
    U1 = b.get_moments("conserved")
    b.run(10 ** 6, 0.03)                   # every tube already at t_end
    assert np.array_equal(b.get_moments("conserved"), U1)
    t, st = b.clock()
    assert np.allclose(t, 0.03, rtol=0, atol=1e-15)
    b.run(10 ** 6, 0.04)
    t, _ = b.clock()
    assert np.allclose(t, 0.04, rtol=0, atol=1e-15)
    d = b.diagnostics()
    assert d["n_nonfinite"] == 0 and d["n_nonpositive"] == 0


def test_mixed_tubes_autotune(mx):
    """The autotuner restores state and clocks, picks a legal shape, and the
    tuned run equals the default-shape run bitwise."""
    tubes = wl.batch_tubes(16, nmin=200, nmax=2000)
    b = sod_batch(mx, tubes)
    U0 = b.get_moments("conserved")
    nt, cl, ms = b.autotune(0.004)
    assert nt in (128, 256) and cl in (1, 2, 4, 8) and ms > 0
    assert np.array_equal(b.get_moments("conserved"), U0)
    t, st = b.clock()
    assert (t == 0).all() and (st == 0).all()
    b.run(10 ** 6, 0.01)
    a = sod_batch(mx, tubes, (128, 1))
    a.run(10 ** 6, 0.01)
    assert np.array_equal(b.get_moments("conserved"), a.get_moments("conserved"))
    print(f"autotuned shape {nt} threads x {cl} CTAs: {ms:.3f} ms over t = 0.004")


@pytest.mark.parametrize("kn", [1e-3, 0.1, 10.0])
def test_mixed_tube_l1_bound(mx, orc, kn):
    """Free run to t = 0.05 against the FP64 oracle, per field, within 10x the
    problem's sensitivity to a 1e-7 relative perturbation of its data."""
    nc, r = 400, 8.0
    prim = wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None]
    cfg = oracle_cfg(orc, nc, kn)
    ref, _, _ = orc.run(cfg, cons_field(orc, prim), 0.0, 0.05, 100000)
    rng = np.random.default_rng(5)
    pert = prim * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=prim.shape))
    alt, _, _ = orc.run(cfg, cons_field(orc, pert), 0.0, 0.05, 100000)
    sens = l1_rel(orc.cons2prim_field(alt), orc.cons2prim_field(ref))
    b = sod_batch(mx, [(nc, kn, r)])
    b.run(10 ** 6, 0.05)
    got = soa_to_aos(b.get_moments("primitive").reshape(14, 1, nc))
    err = l1_rel(got, orc.cons2prim_field(ref))
    act = [0, 1, 4, 7, 9, 10, 13]          # fields that are not identically zero in 1D
    bound = np.maximum(10 * sens[act], 1e-12)
    print(f"Kn={kn}: mixed L1 {err[act].max():.2e}, sensitivity {sens[act].max():.2e}")
    assert (err[act] <= bound).all(), (err[act], sens[act])
    for k in sorted(set(range(14)) - set(act)):
        assert err[k] == 0.0 or np.abs(got[..., k]).max() == 0.0


def test_mixed_tubes_config_batch(mx, orc):
    """The full 256-tube batch (512..8192 cells) to t = 0.2 in one graph
    launch: every tube reaches t_end with a finite, realizable state; the
    smallest tube matches the FP64 oracle within the L1 bound."""
    tubes = wl.batch_tubes()
    b = sod_batch(mx, tubes)
    b.autotune(0.002)
    b.run(10 ** 7, 0.2)
    t, st = b.clock()
    assert np.allclose(t, 0.2, rtol=0, atol=1e-14)
    d = b.diagnostics()
    assert d["n_nonfinite"] == 0 and d["n_nonpositive"] == 0 and d["n_sigma_above_one"] == 0
    i = int(np.argmin([nc for (nc, kn, r) in tubes]))
    nc, kn, r = tubes[i]
    prim = wl.sod_prim(14, nc, rhoR=1 / r, PR=1 / r)[None]
    cfg = oracle_cfg(orc, nc, kn)
    ref, _, _ = orc.run(cfg, cons_field(orc, prim), 0.0, 0.2, 10 ** 6)
    rng = np.random.default_rng(6)
    pert = prim * (1 + 1e-7 * rng.choice([-1.0, 1.0], size=prim.shape))
    alt, _, _ = orc.run(cfg, cons_field(orc, pert), 0.0, 0.2, 10 ** 6)
    sens = l1_rel(orc.cons2prim_field(alt), orc.cons2prim_field(ref))
    got = soa_to_aos(b.unpack(b.get_moments("primitive"))[i][:, None, :])
    err = l1_rel(got, orc.cons2prim_field(ref))
    act = [0, 1, 4, 7, 9, 10, 13]
    print(f"smallest tube ({nc} cells, Kn={kn:.3g}): L1 {err[act].max():.2e}, "
          f"sensitivity {sens[act].max():.2e}; steps {st.min()}..{st.max()}")
    assert (err[act] <= np.maximum(10 * sens[act], 1e-12)).all(), (err[act], sens[act])
