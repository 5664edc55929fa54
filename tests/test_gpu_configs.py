"""The workload configurations at their full sizes and end times, through the
C ABI: the 512^2 isentropic vortex over one period (FP64 and FP32, error
against the exact solution, FP32 against FP64, conservation), the 4096x1024
Mach-10 double Mach reflection to t = 0.2 (positivity and the MOOD flag
fraction every step), and the 64 uneven four-quadrant problems to t = 0.25
(FP32 against FP64 per problem)."""
import os

import numpy as np
import pytest

import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GAMMA = 1.4
# the 64-problem batch to t = 0.25 in FP64 and FP32 takes about 20 minutes of
# a GPU: it runs when GPMOOD_LONG_TESTS=1; the shorter FP32-against-FP64
# batch check to t = 0.02 and everything else always run
LONG = os.environ.get("GPMOOD_LONG_TESTS") == "1"
long_only = pytest.mark.skipif(not LONG, reason="set GPMOOD_LONG_TESTS=1 (minutes of GPU time)")


def pressure(U):
    return (GAMMA - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])


_vortex = {}


def vortex_period(precision):
    if precision not in _vortex:
        p = I.vortex(n=512, R=3)
        g = gp.GPMood(p, precision)
        g.set_state(p["U0"])
        n = g.run(10.0)
        _vortex[precision] = (g.get_state(), n, g.flags(maps=False)[2]["t"])
        g.close()
    return _vortex[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vortex_512_one_period(precision):
    """One period (t = 10) of the vortex on [-5,5]^2 at 512^2: the L1
    density error against the exact (translated) solution, and the totals of
    all four conserved variables (periodic: no boundary flux) to round-off
    per step -- the stage accumulation is FP64 on both paths."""
    p = I.vortex(n=512, R=3)
    U, n, t = vortex_period(precision)
    assert abs(t - 10.0) < 1e-12
    ex = I.vortex(n=512, R=3, t=10.0)["U0"]
    dA = (10.0 / 512) ** 2
    L1 = float(np.abs(U[0] - ex[0]).sum() * dA)
    drift = [abs(U[v].sum() - p["U0"][v].sum()) / np.abs(p["U0"][v]).sum() for v in range(4)]
    print(f"{precision}: {n} steps to t = 10, L1 density error vs exact {L1:.4e}, "
          f"relative drift of the totals {['%.1e' % d for d in drift]}")
    assert L1 < 1e-3
    assert max(drift) <= 1e-13 * n
    assert U[0].min() > 0 and pressure(U).min() > 0


def test_vortex_512_fp32_against_fp64():
    """FP32 reconstruction / flux / detection against the FP64 path after one
    period: float rounding of the face fluxes (6e-8 relative) over about
    5,800 stages stays near 1e-6 in the mean."""
    U64, n64, _ = vortex_period("fp64")
    U32, n32, _ = vortex_period("fp32")
    d = float(np.abs(U32[0] - U64[0]).mean())
    print(f"FP32 vs FP64 after one period: mean |drho| {d:.3e}, steps {n32} / {n64}")
    assert abs(n32 - n64) <= 1
    assert d <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dmr_full_size_to_t_end(precision):
    """4096 x 1024 to t = 0.2.  Every step: no FOG candidate failed PAD in
    any stage (the certificate that every stage output is admissible, the
    RK combinations being convex), and the first-pass flag fraction per
    stage is logged; the state itself is checked for positivity every 400
    steps and at the end.  Last FP64 run: 5712 steps, largest first-pass
    flag fraction 0.39% of the cells; FP32: 5680 steps, 0.41%."""
    p = I.dmr(nx=4096, ny=1024, R=3)
    g = gp.GPMood(p, precision)
    g.set_state(p["U0"])
    ncell = 4096 * 1024
    fr, t, k = [], 0.0, 0
    while t < 0.2 * (1 - 1e-14):
        st = g.flags(maps=False)[2]
        last_dt = st["dt"]
        if 0.2 - t < 2.0 * last_dt:
            g.run(0.2)
        else:
            g.step()
        st = g.flags(maps=False)[2]
        t = st["t"]
        k += 1
        assert st["nfog_pad"] == [0, 0, 0], (k, st["nfog_pad"])
        fr.append([b / ncell for b in st["nbad_first"]])
        if k % 400 == 0:
            U = g.get_state()
            assert U[0].min() > 0 and pressure(U).min() > 0, k
    U = g.get_state()
    g.close()
    fr = np.array(fr)
    print(f"{precision}: {len(fr)} steps to t = 0.2; first-pass flag fraction per stage: "
          f"max {fr.max():.4f}, mean {fr.mean():.4f}, last step {fr[-1].round(4).tolist()}")
    assert U[0].min() > 0 and pressure(U).min() > 0
    assert np.isfinite(U).all()
    assert fr.max() < 0.10


@long_only
def test_batch_64_quadrants_to_t_end_fp32_against_fp64():
    """The 64 uneven four-quadrant problems (128^2 .. 1024^2, seed 0) to
    t = 0.25 in one batch, FP64 and FP32: every problem reaches t_end with
    positive density and pressure; the FP32 path's mean density difference
    from the FP64 path is stated per problem (shocks move MOOD decisions, so
    the difference is that of two schemes, not of rounding alone)."""
    probs = I.quadrant_batch(count=64, seed=0)
    res = {}
    for precision in ("fp64", "fp32"):
        b = gp.GPMoodBatch(probs, precision)
        b.set_state([q["U0"] for q in probs])
        b.run(0.25)
        t, dt, ns, _ = b.info()
        np.testing.assert_allclose(t, 0.25, rtol=1e-13)
        res[precision] = b.get_state()
        b.close()
    diffs = []
    for k, q in enumerate(probs):
        U64, U32 = res["fp64"][k], res["fp32"][k]
        for U in (U64, U32):
            assert U[0].min() > 0 and pressure(U).min() > 0, k
        diffs.append(float(np.abs(U32[0] - U64[0]).mean() / np.abs(U64[0]).mean()))
    diffs = np.array(diffs)
    print(f"FP32 vs FP64, relative mean |drho| per problem: median {np.median(diffs):.2e}, "
          f"max {diffs.max():.2e}")
    assert diffs.max() < 1e-2


def test_batch_64_quadrants_fp32_against_fp64_early():
    """The 64-problem batch to t = 0.02 (about 170 steps of the 1024^2
    problems) in FP64 and FP32: the FP32 path's relative mean density
    difference from the FP64 path, per problem, before the shocks have
    moved many MOOD decisions apart."""
    probs = I.quadrant_batch(count=64, seed=0)
    res = {}
    for precision in ("fp64", "fp32"):
        b = gp.GPMoodBatch(probs, precision)
        b.set_state([q["U0"] for q in probs])
        b.run(0.02)
        t, dt, ns, _ = b.info()
        np.testing.assert_allclose(t, 0.02, rtol=1e-13)
        res[precision] = b.get_state()
        b.close()
    diffs = np.array([float(np.abs(res["fp32"][k][0] - res["fp64"][k][0]).mean()
                            / np.abs(res["fp64"][k][0]).mean()) for k in range(len(probs))])
    for k in range(len(probs)):
        U = res["fp32"][k]
        assert U[0].min() > 0 and pressure(U).min() > 0, k
    print(f"batch FP32 vs FP64 at t = 0.02, relative mean |drho| per problem: median "
          f"{np.median(diffs):.2e}, largest {diffs.max():.2e}")
    assert diffs.max() < 1e-3


@pytest.mark.parametrize("seed", [5, 11])
def test_fp32_mood_iterations_follow_fp64(seed):
    """A 1024^2 four-quadrant problem over 20 steps in FP64 and in FP32: the
    MOOD iteration counts of the FP32 path stay within twice those of the
    FP64 path, and the first-pass troubled maps of the first step agree; the
    maps of later steps are compared and their mismatch count is reported.
    Long loops (hundreds of iterations on seed 11) occur in both precisions
    and in the oracle alike: along a discontinuity that lies on a grid line,
    lowering one cell changes the EDP1 radius of the face it shares with its
    neighbour, whose state on that face then fails the face-state check, so
    the lowering walks along the line one cell per iteration."""
    p = I.quadrants(n=1024, R=3, seed=seed)
    its, firsts = {}, {}
    for precision in ("fp64", "fp32"):
        g = gp.GPMood(p, precision)
        g.set_state(p["U0"])
        it, fm = [], []
        for _ in range(20):
            g.step()
            _, first, st = g.flags()
            it.append(st["iters"])
            fm.append(first)
        g.close()
        its[precision], firsts[precision] = np.array(it), fm
    mism = [int((a != b).sum()) for a, b in zip(firsts["fp32"], firsts["fp64"])]
    print(f"seed {seed}: max iterations per stage FP64 {its['fp64'].max()}, FP32 "
          f"{its['fp32'].max()}; summed {its['fp64'].sum()} / {its['fp32'].sum()}; first-pass "
          f"map mismatches per step {mism}")
    assert mism[0] == 0
    assert its["fp32"].max() <= 2 * its["fp64"].max()
    assert its["fp32"].sum() <= 2 * its["fp64"].sum()
