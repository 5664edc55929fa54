"""Batches of independent problems of uneven sizes (gpmood_batch_*) against
single-problem handles running the same kernels, and against the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(4))


def mixed_problems(R=3):
    # uneven grids sharing ell/dx = 12: shocks (MOOD active) and a smooth wave
    states = I.quadrant_states(seed=4, count=3)
    probs = [I.quadrants(n=40, ny=40, R=R, states=states[0]),
             I.quadrants(n=72, ny=72, R=R, states=states[1]),
             I.quadrants(n=33, ny=33, R=R, states=states[2])]
    w = I.density_wave(nx=48, ny=48, amp=0.2, R=R, ell=12.0 / 48)
    probs.append(w)
    return probs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_handles(precision):
    probs = mixed_problems()
    b = gp.GPMoodBatch(probs, precision)
    b.set_state([q["U0"] for q in probs])
    singles = [gp.GPMood(q, precision) for q in probs]
    for s, q in zip(singles, probs):
        s.set_state(q["U0"])
    for _ in range(3):
        b.step()
        for s in singles:
            s.step()
    Ub = b.get_state()
    t, dt, ns, st = b.info()
    # the same device functions compiled into two kernels: FP64 agrees to
    # round-off, FP32 to float rounding (contraction can differ per kernel)
    tol = 1e-13 if precision == "fp64" else 1e-5
    for k, s in enumerate(singles):
        Us = s.get_state()
        assert relerr(Ub[k], Us) <= tol, k
        _, _, ss = s.flags(maps=False)
        assert abs(t[k] - ss["t"]) <= (1e-14 if precision == "fp64" else 1e-6) * ss["t"]
    assert sum(st["nbad_first"]) > 0  # the MOOD loop ran inside the batch
    # the autotuner's choices: the fused x+y face kernel (warps [0, 0]) or one
    # sweep per direction with 4 or 8 warps, and the update and MOOD grids
    w, nb = b.tuning()
    assert (w == [0, 0] or all(x in (4, 8) for x in w)) and all(x > 0 for x in nb)
    up, mood = b.grids()
    assert up > 0 and mood > 0


def test_batch_first_step_against_oracle():
    probs = mixed_problems()
    b = gp.GPMoodBatch(probs)
    b.set_state([q["U0"] for q in probs])
    b.step()
    Ub = b.get_state()
    for k, q in enumerate(probs):
        Uo, so, _, _ = O.Oracle(q).step(q["U0"], 0.0)
        assert relerr(Ub[k], Uo) <= 1e-11, k


def test_batch_run_reaches_t_end_per_problem():
    probs = mixed_problems(R=2)
    b = gp.GPMoodBatch(probs)
    b.set_state([q["U0"] for q in probs])
    t_end = 0.02
    b.run(t_end)
    t, dt, ns, _ = b.info()
    np.testing.assert_allclose(t, t_end, rtol=1e-13)
    Ub = b.get_state()
    for k, q in enumerate(probs):
        s = gp.GPMood(q)
        s.set_state(q["U0"])
        n = s.run(t_end)
        assert n == ns[k]
        assert relerr(Ub[k], s.get_state()) <= 1e-13


def test_batch_eager_launches_equal_the_step_graph():
    probs = mixed_problems()
    out = []
    for eager in (False, True):
        b = gp.GPMoodBatch(probs, "fp64", eager=eager)
        b.set_state([q["U0"] for q in probs])
        for _ in range(3):
            b.step()
        out.append((b.get_state(), b.info()))
        b.close()
    (U0, i0), (U1, i1) = out
    for k in range(len(probs)):
        assert np.array_equal(U0[k], U1[k]), k
    assert list(i0[0]) == list(i1[0])
    assert i0[3]["iters"] == i1[3]["iters"]
