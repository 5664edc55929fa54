"""Pins of the oracle's POL-MOOD3 (Sec. 3.1 (iv), eq. poly3, eq. p3_coeffs,
App. C) and of the Shu-Osher shock tube (Sec. 5.2.1): the printed Riemann-state
weights of Poly3, exactness on quadratics, the cell mean, the third-order
rate of the full scheme, the printed Table 2 entry and the printed Shu-Osher
peaks, with and without CSD."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_08683_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
G2 = 0.5 / math.sqrt(3.0)  # two-point Gauss abscissa on [-1/2, 1/2]


def _gold(name):
    return json.load(open(os.path.join(GOLD, name)))


# stencil order of the oracle (App. A labels): centre, west, north, east, south
OFF = [(0, 0), (-1, 0), (0, 1), (1, 0), (0, -1)]


def _weights_at(xs, ys, dim=2):
    n = 5 if dim == 2 else 3
    out = np.zeros(n)
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        out[m] = O.poly3_eval(dim, e, xs, ys)
    return out


def test_stencil_labels_are_app_a():
    assert [tuple(r) for r in O.stencil(2, 1)] == OFF


def test_east_face_weights_are_the_printed_ones():
    gold = _gold("poly3_face_weights.json")
    np.testing.assert_allclose(_weights_at(0.5, G2), gold["east_g1"], rtol=0, atol=2e-16)
    np.testing.assert_allclose(_weights_at(0.5, -G2), gold["east_g2"], rtol=0, atol=2e-16)


def test_other_faces_are_the_rotated_expressions():
    # the west / north / south weights are the east ones with the stencil
    # mirrored or rotated (the paper rotates the printed expressions)
    gold = np.array(_gold("poly3_face_weights.json")["east_g1"])
    east = {OFF[m]: gold[m] for m in range(5)}
    for face, (xs, ys), rot in (
        ("west", (-0.5, -G2), lambda a, b: (-a, -b)),
        ("north", (-G2, 0.5), lambda a, b: (-b, a)),
        ("south", (G2, -0.5), lambda a, b: (b, -a)),
    ):
        w = _weights_at(xs, ys)
        for m, (a, b) in enumerate(OFF):
            # the stencil cell (a, b) plays the role of east's rotated-back cell
            src = [k for k in east if rot(*k) == (a, b)][0]
            assert abs(w[m] - east[src]) < 2e-16, (face, (a, b))


def _cell_means(c, dim):
    """exact means over the unit cells of f = c0 + c1 x + c2 x^2 + c3 y + c4 y^2 + c5 xy"""
    offs = OFF if dim == 2 else [(0, 0), (-1, 0), (1, 0)]
    v = 1.0 / 12.0
    return np.array([c[0] + c[1] * a + c[2] * (a * a + v) + c[3] * b + c[4] * (b * b + v)
                     + c[5] * a * b for a, b in offs])


@pytest.mark.parametrize("seed", range(4))
def test_exact_on_quadratics(seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2, 2, 6)
    qv = _cell_means(c, 2)
    for xs, ys in rng.uniform(-0.5, 0.5, (8, 2)):
        f = c[0] + c[1] * xs + c[2] * xs * xs + c[3] * ys + c[4] * ys * ys
        # the xy monomial has zero mean on all five cells: Poly3 cannot see it
        assert abs(O.poly3_eval(2, qv, xs, ys) - f) < 1e-13
    c1 = c.copy()
    c1[3:] = 0.0
    q1 = _cell_means(c1, 1)
    for xs in rng.uniform(-0.5, 0.5, 4):
        f = c1[0] + c1[1] * xs + c1[2] * xs * xs
        assert abs(O.poly3_eval(1, q1, xs, 0.0) - f) < 1e-13


def test_poly3_keeps_the_cell_mean():
    # the 2x2 Gauss rule integrates the quadratic exactly over the centre cell
    rng = np.random.default_rng(5)
    qv = rng.uniform(0.5, 2.0, 5)
    mean = np.mean([O.poly3_eval(2, qv, a, b) for a in (G2, -G2) for b in (G2, -G2)])
    assert abs(mean - qv[0]) < 1e-15


def test_curvature_is_poly3_second_derivative():
    # POL-MOOD3's u2 curvature: p3's second derivative, exact on the cell
    # averages of a cubic (centred second difference of cubic averages)
    p = I.uniform(12, 10, R=1, state=(1.0, 0.0, 0.0, 1.0), bc="outflow")
    p["cascade"], p["recon"] = [1, 0], "poly3"
    o = O.Oracle(p)
    H, dx, dy = o.H, (p["x1"] - p["x0"]) / 12, (p["y1"] - p["y0"]) / 10
    Xg = o.fill_ghosts(p["U0"])
    jj, ii = np.meshgrid(np.arange(-H, 10 + H), np.arange(-H, 12 + H), indexing="ij")
    x, y = ii * dx, jj * dy  # cell centres in physical units

    def cube_mean(s, h):  # mean of s^3 over [s - h/2, s + h/2]
        return s ** 3 + s * h * h / 4.0

    Xg[0] = 2.0 + 0.3 * cube_mean(x, dx) - 0.7 * cube_mean(y, dy) + 0.1 * x * y
    for i, j in ((3, 4), (7, 2), (10, 8)):
        assert abs(o.curvature(Xg, 0, i, j) - 0.3 * 6 * i * dx) < 1e-8
        assert abs(o.curvature(Xg, 1, i, j) + 0.7 * 6 * j * dy) < 1e-8


def test_polmood3_rejects_other_cascades():
    p = I.vortex(n=16, R=2)
    p["recon"] = "poly3"
    with pytest.raises(RuntimeError):
        O.Oracle(p)


def test_polmood3_full_scheme_is_third_order():
    amp, errs = 0.1, []
    for n in (16, 32):
        p = I.density_wave(n=n, amp=amp, R=1, ell=0.1)
        p["recon"] = "poly3"
        o = O.Oracle(p)
        dt = 0.3 / n
        t_end = 0.1
        nst = int(math.ceil(t_end / dt))
        dt = t_end / nst
        U = p["U0"]
        for k in range(nst):
            U, st, _, _ = o.step(U, k * dt, dt_fixed=dt)
        ex = I.density_wave(n=n, amp=amp, R=1, ell=0.1, t=t_end)["U0"]
        errs.append(np.abs(U[0] - ex[0]).mean())
    eoc = math.log2(errs[0] / errs[1])
    assert eoc > 2.4, (errs, eoc)


@pytest.mark.slow
def test_table2_polmood3_at_50():
    """Table 2's POL-MOOD3 entry at N = 50 is met to 5e-7 relative with
    SSP-RK3 at CFL 0.5; at the CFL 0.8 stated for the runs, the error is 0.8%
    larger (the time error of this scheme grows with the CFL number)."""
    gold = _gold("table2_polmood3.json")
    p = I.vortex(n=50, lo=0.0, hi=20.0, R=1, ell=1.0, cascade=[1, 0])
    p["recon"] = "poly3"
    ex = I.vortex(n=50, lo=0.0, hi=20.0, R=1, ell=1.0, t=20.0)["U0"]
    o = O.Oracle(p)
    L1 = {}
    for cfl in (0.5, 0.8):
        U, _, _ = o.run(p["U0"], 20.0, cfl=cfl)
        L1[cfl] = np.abs(U[0] - ex[0]).sum() * 0.4 ** 2
    assert abs(L1[0.5] - gold["L1"][0]) < 2e-6 * gold["L1"][0], L1
    assert 0.0 < L1[0.8] - gold["L1"][0] < 0.01 * gold["L1"][0], L1


def _shu_peak(scheme, csd_on=1, n=256):
    p = I.shu_osher(n=n, scheme=scheme, csd_on=csd_on)
    U, _, t = O.Oracle(p).run(p["U0"], 1.8)
    x = (np.arange(n) + 0.5) * 9.0 / n
    r = U[0, 0]
    k = int(np.argmax(r))
    return r[k], x[k], r


def test_shu_osher_peaks_follow_the_paper():
    gold = _gold("shu_osher_peaks.json")
    got = {}
    for scheme in ("GP-MOOD3", "POL-MOOD3", "GP-MOOD5", "GP-MOOD7"):
        rho, x, r = _shu_peak(scheme)
        got[scheme] = rho
        assert abs(x - gold["x_peak"]) < 0.03, (scheme, x)
        assert abs(rho - gold["rho_max"][scheme]) < 0.05, (scheme, rho)
        assert np.isfinite(r).all() and r.min() > 0
    # the order the paper reports: the GP-MOOD5/7 pair, then GP-MOOD3, then POL-MOOD3
    assert min(got["GP-MOOD5"], got["GP-MOOD7"]) > got["GP-MOOD3"] + 0.2 > got["POL-MOOD3"] + 0.2


def test_shu_osher_without_csd_is_more_diffusive():
    # Sec. 5.2.1: without CSD every peak drops; GP-MOOD5 loses most of its
    # lead over GP-MOOD3 (with CSD: +0.27; without: about half of it is lost)
    on = {s: _shu_peak(s)[0] for s in ("GP-MOOD3", "GP-MOOD5")}
    off = {s: _shu_peak(s, csd_on=0)[0] for s in ("GP-MOOD3", "GP-MOOD5", "POL-MOOD3")}
    assert off["GP-MOOD3"] < on["GP-MOOD3"] and off["GP-MOOD5"] < on["GP-MOOD5"] - 0.08
    assert off["GP-MOOD5"] - on["GP-MOOD3"] < 0.6 * (on["GP-MOOD5"] - on["GP-MOOD3"])
    assert off["POL-MOOD3"] < off["GP-MOOD3"]


def test_shu_osher_set_up():
    # Sec. 5.2.1: the Mach 3 shock at x = 0.5 on [0, 9], the sinusoid ahead of
    # it at rest under unit pressure; cell averages of the printed states
    p = I.shu_osher(n=256, scheme="GP-MOOD7")
    U = p["U0"][:, 0, :]
    dx = 9.0 / 256
    x = (np.arange(256) + 0.5) * dx
    left = x < 0.5 - dx
    assert np.allclose(U[0][left], 3.857143) and np.allclose(U[1][left], 3.857143 * 2.629369)
    right = x > 0.5 + dx
    # the average of 1 + 0.2 sin(5 (x - 4.5)) over a cell, by the exact integral
    lo, hi = x[right] - dx / 2, x[right] + dx / 2
    mean = 1.0 + 0.2 * (np.cos(5 * (lo - 4.5)) - np.cos(5 * (hi - 4.5))) / (5 * dx)
    assert np.abs(U[0][right] - mean).max() < 1e-12
    assert np.abs(U[1][right]).max() == 0.0 and np.allclose(U[3][right], 1.0 / 0.4)
    assert p["bc"][:2] == ["dirichlet", "outflow"] and p["t_end"] == 1.8
    assert abs(p["ell"] - 6 * dx) < 1e-15 and p["rk"] == 4 and p["cascade"] == [3, 1, 0]
    assert abs(p["cfl"] - 0.8 * dx ** 0.75) < 1e-15  # Delta^((2R+1)/4 - 1), R = 3
