"""POL-MOOD3 (Sec. 3.1 (iv)) and the Shu-Osher shock tube (Sec. 5.2.1)
through the C ABI: POL-MOOD3 steps locked to the oracle in 2D and 1D, the four
schemes of the paper on the Shu-Osher tube with and without CSD against the
oracle (locked steps, then free runs to t = 1.8), the printed peak densities,
the 4096-cell reference solution, and the POL-MOOD3 column of Table 2."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SCHEMES = ("GP-MOOD3", "POL-MOOD3", "GP-MOOD5", "GP-MOOD7")


def _gold(name):
    return json.load(open(os.path.join(GOLD, name)))


def relerr(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(4))


def locked_steps(p, nsteps, tol, U=None, t=0.0, precision="fp64"):
    """nsteps steps of the CUDA path, each from the oracle's state, against
    the oracle's step: dt, first-pass flags, final radii, iteration counts."""
    g, o = gp.GPMood(p, precision), O.Oracle(p)
    U = p["U0"].copy() if U is None else U
    flagged = 0
    for k in range(nsteps):
        g.set_state(U)
        g.set_time(t)
        dtg = g.step(want_dt=True)
        Ug = g.get_state()
        og, bg, sg = g.flags()
        Uo, st, oo, bo = o.step(U, t)
        # the FP32 path takes its CFL rate in float (a few 1e-7 relative)
        assert abs(dtg - st["dt"]) <= (1e-14 if precision == "fp64" else 1e-6) * st["dt"], k
        if precision == "fp64":
            assert (bg == bo).all() and (og == oo).all(), k
            assert sg["iters"] == st["iters"], k
        assert relerr(Ug, Uo) <= tol, (k, relerr(Ug, Uo))
        flagged += sum(st["nbad_first"])
        U, t = Uo, t + st["dt"]
    g.close()
    return flagged


def test_polmood3_quadrants_locked_to_oracle():
    p = I.quadrants(n=48, ny=40, R=1, seed=3, cascade=[1, 0])
    p["recon"] = "poly3"
    assert locked_steps(p, 4, 1e-12) > 0


def test_polmood3_fp32_quadrants_close_to_oracle():
    p = I.quadrants(n=48, ny=40, R=1, seed=3, cascade=[1, 0])
    p["recon"] = "poly3"
    locked_steps(p, 2, 2e-5, precision="fp32")


def test_polmood3_needs_radius_one_and_single_handles():
    p = I.quadrants(n=32, R=2, seed=3)
    p["recon"] = "poly3"
    with pytest.raises(gp.GpmoodError):
        gp.GPMood(p)
    q = I.quadrants(n=32, R=1, seed=3, cascade=[1, 0])
    q["recon"] = "poly3"
    with pytest.raises(gp.GpmoodError):
        gp.GPMoodBatch([q, q])


def _oracle_run(p, t_end):
    o = O.Oracle(p)
    U, n, t = o.run(p["U0"], t_end)
    return U, n


@pytest.mark.parametrize("csd_on", [1, 0])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_shu_osher_locked_to_oracle(scheme, csd_on):
    """Ten steps from the initial state and ten from the oracle's state at
    t = 0.9, where the shock runs through the sinusoid."""
    p = I.shu_osher(n=256, scheme=scheme, csd_on=csd_on)
    assert locked_steps(p, 10, 1e-12) > 0
    Um, _ = _oracle_run(p, 0.9)
    assert locked_steps(p, 10, 1e-12, U=Um, t=0.9) > 0


def _peak(U):
    n = U.shape[-1]
    r = U[0, 0]
    k = int(np.argmax(r))
    return float(r[k]), (k + 0.5) * 9.0 / n


@pytest.mark.parametrize("csd_on", [1, 0])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_shu_osher_run_to_t_end_against_oracle(scheme, csd_on):
    """The full run to t = 1.8: the CUDA path's density profile within 1e-9
    (L1, FP64) of the oracle's, the same step count, and the peak where the
    paper measures it."""
    p = I.shu_osher(n=256, scheme=scheme, csd_on=csd_on)
    g = gp.GPMood(p)
    g.set_state(p["U0"])
    ng = g.run(1.8)
    Ug = g.get_state()
    g.close()
    Uo, no = _oracle_run(p, 1.8)
    L1 = np.abs(Ug[0, 0] - Uo[0, 0]).mean()
    rg, xg = _peak(Ug)
    ro, _ = _peak(Uo)
    print(f"{scheme} CSD {'on' if csd_on else 'off'}: {ng} steps, peak rho {rg:.4f} at x = {xg:.3f}"
          f" (oracle {ro:.4f}); L1 density difference {L1:.2e}")
    assert ng == no
    assert L1 <= 1e-9, L1
    assert abs(xg - 6.34) < 0.03


def test_shu_osher_peaks_and_fp32():
    gold = _gold("shu_osher_peaks.json")["rho_max"]
    got = {}
    for scheme in SCHEMES:
        p = I.shu_osher(n=256, scheme=scheme)
        for precision in ("fp64", "fp32"):
            g = gp.GPMood(p, precision)
            g.set_state(p["U0"])
            g.run(1.8)
            got[scheme, precision] = _peak(g.get_state())[0]
            g.close()
        print(f"{scheme}: peak rho {got[scheme, 'fp64']:.4f} (FP32 {got[scheme, 'fp32']:.4f}), "
              f"printed {gold[scheme]}")
        assert abs(got[scheme, "fp64"] - gold[scheme]) < 0.05
        # float rounding can move a MOOD decision at the peak (GP-MOOD7: one
        # part in 4000), well inside the two printed digits
        assert abs(got[scheme, "fp32"] - got[scheme, "fp64"]) < 2e-3


def test_shu_osher_reference_solution():
    """POL-MOOD3 with SSP-RK3 on 4096 cells, the paper's reference: peak 4.69."""
    gold = _gold("shu_osher_peaks.json")["rho_max"]["reference_4096"]
    p = I.shu_osher(n=4096, scheme="POL-MOOD3")
    g = gp.GPMood(p)
    g.set_state(p["U0"])
    ns = g.run(1.8)
    rho, x = _peak(g.get_state())
    g.close()
    print(f"reference POL-MOOD3 4096 cells: {ns} steps, peak rho {rho:.4f} at x = {x:.4f}")
    assert abs(rho - gold) < 0.015 and abs(x - 6.34) < 0.01


@pytest.mark.slow
def test_table2_polmood3_column():
    """Table 2's POL-MOOD3 column (vortex on [0,20]^2 to t = 20, SSP-RK3):
    at the stated CFL 0.8 every L1 error is within 1% of the printed one and
    every EOC within 0.02 of the printed EOC.  The printed errors do not come
    from one constant CFL number: N = 50 is met to 2e-6 at CFL 0.5, and the
    other resolutions fall at growing CFL numbers (about 0.59, 0.71, and
    above 0.8 at N = 400), so the 1% band is the time error's share."""
    gold = _gold("table2_polmood3.json")
    errs = []
    for k, n in enumerate(gold["N"]):
        ex = I.vortex(n=n, lo=0.0, hi=20.0, R=1, ell=1.0, t=20.0)["U0"]
        p = I.vortex(n=n, lo=0.0, hi=20.0, R=1, ell=1.0, cascade=[1, 0])
        p["recon"] = "poly3"
        g = gp.GPMood(p)
        g.set_state(p["U0"])
        g.run(20.0)
        L1 = float(np.abs(g.get_state()[0] - ex[0]).sum() * (20.0 / n) ** 2)
        if n == 50:
            g.set_state(p["U0"])
            g.set_time(0.0)
            g.run(20.0, cfl=0.5)
            L1_05 = float(np.abs(g.get_state()[0] - ex[0]).sum() * 0.4 ** 2)
            assert abs(L1_05 - gold["L1"][0]) < 2e-6 * gold["L1"][0], L1_05
        g.close()
        errs.append(L1)
        print(f"POL-MOOD3 N={n}: L1 {L1:.8e} (printed {gold['L1'][k]:.8e}, "
              f"ratio {L1 / gold['L1'][k]:.5f})")
        assert abs(L1 - gold["L1"][k]) < 0.01 * gold["L1"][k], (n, L1)
    for k in range(1, 4):
        eoc = math.log(errs[k - 1] / errs[k]) / math.log(2.0)
        print(f"POL-MOOD3 EOC {eoc:.3f} (printed {gold['EOC'][k]})")
        assert abs(eoc - gold["EOC"][k]) < 0.02, (k, eoc)
