"""The Mach-10 double Mach reflection at its full size (4096 x 1024, GP-R3
cascade 7->5->3->1), FP64 and FP32, through the C ABI: ten steps with
positivity of density and pressure checked after every step and the
first-pass MOOD flag fraction of every stage recorded; the FP32 path against
the FP64 path; and a reduced grid run to the full t_end against the oracle.
Outflow, inflow and a moving top boundary leave no conservation invariant."""
import functools

import numpy as np
import pytest

import oracle as O
import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@functools.lru_cache(maxsize=1)
def dmr_full():
    return I.dmr(nx=4096, ny=1024, R=3)


def pressure(U):
    return (GAMMA - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])


@functools.lru_cache(maxsize=2)
def ten_steps(precision):
    p = dmr_full()
    g = gp.GPMood(p, precision)
    g.set_state(p["U0"])
    n = p["nx"] * p["ny"]
    fractions, minima = [], []
    for _ in range(10):
        g.step()
        _, _, st = g.flags(maps=False)
        fractions.append([b / n for b in st["nbad_first"]])
        U = g.get_state()
        minima.append((float(U[0].min()), float(pressure(U).min())))
    t = g.flags(maps=False)[2]["t"]
    U = g.get_state()
    g.close()
    return U, fractions, minima, t


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dmr_full_size_ten_steps_positive_with_flag_fractions(precision):
    U, fractions, minima, t = ten_steps(precision)
    for k, (rmin, pmin) in enumerate(minima):
        assert rmin > 0.0 and pmin > 0.0, (k, rmin, pmin)
    f = np.array(fractions)
    print(f"{precision}: first-pass flagged fraction per step and stage:\n{f}")
    # MOOD acts along the shocks only: a thin band of the grid
    assert (f > 0).all() and (f < 0.05).all(), f
    assert np.isfinite(U).all() and t > 0.0


def test_dmr_full_size_fp32_against_fp64():
    U64, _, _, t64 = ten_steps("fp64")
    U32, _, _, t32 = ten_steps("fp32")
    # the FP32 path computes its CFL rate in float: a few 1e-7 relative per step
    assert abs(t32 - t64) <= 5e-6 * t64
    n = U64.shape[1] * U64.shape[2]
    L1 = np.abs(U32[0] - U64[0]).sum() / n
    print(f"FP32 vs FP64 L1 density difference after 10 steps: {L1:.3e}")
    assert L1 <= 1e-4, L1


def test_dmr_reduced_grid_to_t_end_against_oracle():
    """128 x 32 to t = 0.2 (the full t_end) beside the FP64 oracle.  Locked:
    at every step the CUDA path steps from the oracle's state and must match
    the oracle's step (<= 1e-12 relative, identical first-pass flags, final
    radii, MOOD iteration counts and dt).  Free: a second handle runs on its
    own; round-off differences are amplified by the flow and by MOOD
    decisions taken on either side of a threshold, so its L1 density
    difference is held to 1e-8 up to t = 0.1 and reported at t_end."""
    p = I.dmr(nx=128, ny=32, R=3)
    locked, free = gp.GPMood(p), gp.GPMood(p)
    o = O.Oracle(p)
    U, t = p["U0"].copy(), 0.0
    free.set_state(U)
    n_steps, L1_end = 0, None
    while t < 0.2 * (1 - 1e-14):
        locked.set_state(U)
        locked.set_time(t)
        dtg = locked.step(want_dt=True)
        Ug = locked.get_state()
        og, bg, sg = locked.flags()
        Uo, st, oo, bo = o.step(U, t)
        assert abs(dtg - st["dt"]) <= 1e-14 * st["dt"], n_steps
        assert (bg == bo).all() and (og == oo).all(), n_steps
        assert sg["iters"] == st["iters"], n_steps
        rel = max(np.abs(Ug[v] - Uo[v]).max() / np.abs(Uo[v]).max() for v in range(4))
        assert rel <= 1e-12, (n_steps, rel)
        free.step()
        U, t = Uo, t + st["dt"]
        n_steps += 1
        L1 = np.abs(free.get_state()[0] - U[0]).mean()
        if t <= 0.1:
            assert L1 <= 1e-8, (n_steps, t, L1)
        L1_end = L1
    print(f"DMR 128x32 to t=0.2: {n_steps} steps locked to the oracle; "
          f"free-running L1 density difference at t_end {L1_end:.3e}")
    Uf = free.get_state()
    assert Uf[0].min() > 0 and pressure(Uf).min() > 0
