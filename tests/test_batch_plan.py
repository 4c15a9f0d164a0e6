"""The division of a tube batch between the team launch and the single-CTA
fill launch (mxe_batch_plan_fill, host-only: no device needed).

The header defines it: tubes in work order, a team of cl CTAs spends
cl * ceil(chunks / cl) CTA passes per step of a tube, one fill CTA `chunks`;
the fill CTAs take the largest tail of the order whose estimated time (its
passes spread over the fill CTAs) stays within the teams' estimate (their
passes over the teams), with no tail tube longer alone than that estimate.
Checked here against that definition by brute force over every tail length,
on seeded random batches and on degenerate cases."""
import math

import numpy as np
import pytest

import paper_2401_15233_gb300 as mx


def brute_force(cells, steps, chunk, cl, teams, fill):
    n = len(cells)
    ch = [math.ceil(c / chunk) for c in cells]
    team = [math.ceil(k / cl) * s / teams for k, s in zip(ch, steps)]
    solo = [k * s for k, s in zip(ch, steps)]
    best = n
    for nA in range(n - 1, 0, -1):
        if fill == 0:
            break
        TA = sum(team[:nA])
        TB = sum(solo[nA:]) / fill
        if TB <= TA * (1 + 1e-12) and max(solo[nA:]) <= TA * (1 + 1e-12):
            best = nA
        else:
            break
    TA, TB = sum(team[:best]), (sum(solo[best:]) / fill if fill else 0.0)
    return best, max(TA, TB)


def batch(seed, n):
    rng = np.random.default_rng(seed)
    cells = np.round(np.exp(rng.uniform(np.log(100), np.log(8192), n))).astype(np.int32)
    steps = cells * rng.uniform(5, 20, n)            # steps grow with the cell count
    order = np.argsort(-(cells * steps), kind="stable")
    return cells[order], steps[order]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(254, 8, 36, 16), (254, 8, 32, 48), (126, 4, 70, 24),
                                   (254, 2, 100, 4)])
def test_plan_matches_definition(seed, shape):
    chunk, cl, teams, fill = shape
    cells, steps = batch(seed, 40 + 37 * seed)
    nA, t = mx.mxe_batch_plan_fill(cells, steps, chunk, cl, teams, fill)
    nB, tB = brute_force(list(cells), list(steps), chunk, cl, teams, fill)
    assert nA == nB
    assert t == pytest.approx(tB, rel=1e-12)
    assert 1 <= nA <= len(cells)


def test_plan_more_fill_ctas_take_no_fewer_tubes():
    cells, steps = batch(7, 200)
    prev = len(cells)
    for fill in (0, 4, 16, 48, 128):
        nA, _ = mx.mxe_batch_plan_fill(cells, steps, 254, 8, 36, fill)
        assert nA <= prev
        prev = nA


def test_plan_degenerate_cases():
    cells, steps = batch(3, 50)
    assert mx.mxe_batch_plan_fill(cells, steps, 254, 8, 36, 0)[0] == 50     # no fill CTAs
    assert mx.mxe_batch_plan_fill(cells[:1], steps[:1], 254, 8, 36, 16)[0] == 1   # one tube
    # equal one-chunk tubes, one step each: the teams' estimate is nA/teams,
    # the fill's (n - nA)/fill; with teams = fill they meet at nA = n/2
    n, teams, fill = 100, 10, 10
    nA, t = mx.mxe_batch_plan_fill(np.full(n, 200), np.ones(n), 254, 8, teams, fill)
    assert nA == 50 and t == pytest.approx(5.0)
    # a tail tube too long alone stays with the teams
    cells = np.array([8000, 8000, 8000, 8000], dtype=np.int32)
    nA, _ = mx.mxe_batch_plan_fill(cells, np.full(4, 1e4), 254, 8, 4, 100)
    assert nA == 4


@pytest.mark.parametrize("bad", [dict(n=0), dict(chunk=0), dict(cl=0), dict(teams=0),
                                 dict(fill=-1), dict(cell=0), dict(step=-1.0),
                                 dict(step=float("nan"))])
def test_plan_rejects_invalid_arguments(bad):
    cells, steps = np.array([300, 200], dtype=np.int32), np.array([10.0, 5.0])
    if "cell" in bad:
        cells[1] = bad["cell"]
    if "step" in bad:
        steps[1] = bad["step"]
    if bad.get("n") == 0:
        cells, steps = cells[:0], steps[:0]
    with pytest.raises(mx.MaxentError) as e:
        mx.mxe_batch_plan_fill(cells, steps, bad.get("chunk", 254), bad.get("cl", 8),
                               bad.get("teams", 4), bad.get("fill", 2))
    assert e.value.status == mx.EINVAL
