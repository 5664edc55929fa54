"""Pins of the oracle's GP building blocks against things other than itself:
the paper's printed tables (App. A, App. C), closed forms, numerical
quadrature of the kernel definitions and a brute-force dense solve."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("R,N", [(1, 5), (2, 13), (3, 25)])
def test_stencil_is_blocky_diamond(R, N):
    # Sec. 2.2: 5 / 13 / 25 cells for R = 1 / 2 / 3, centre first
    off = O.stencil(2, R)
    assert off.shape == (N, 2)
    assert tuple(off[0]) == (0, 0)
    pts = {tuple(p) for p in off}
    assert len(pts) == N
    assert pts == {(a, b) for a in range(-R, R + 1) for b in range(-R, R + 1) if abs(a) + abs(b) <= R}


def test_appendix_a_delta_tables():
    # App. A: Delta_{mn,d} = e_d.(x_n - x_m)/Delta_d for the R=1 stencil and g1
    gold = _gold("appA_delta_tables.json")
    off = O.stencil(2, 1).astype(float)
    g, _ = O.gauss_rule(2)
    pts = list(off) + [np.array([0.5, g[0]])]  # g1 on the east face, y = +dy/(2 sqrt 3)
    for d, key in ((0, "delta_x"), (1, "delta_y")):
        tab = np.array(gold[key])
        ours = np.array([[pts[n][d] - pts[m][d] for m in range(6)] for n in range(6)])
        np.testing.assert_allclose(ours, tab, atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_gauss_rules_exact_to_degree_2q_minus_1(q):
    # Table QR: q-point rules on [-1/2,1/2] integrate x^k exactly for k <= 2q-1
    g, w = O.gauss_rule(q)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 * 0.5 ** (k + 1) / (k + 1)
        assert abs(np.sum(w * g**k) - exact) < 1e-15
    k = 2 * q
    exact = 2.0 * 0.5 ** (k + 1) / (k + 1)
    assert abs(np.sum(w * g**k) - exact) > 1e-8


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w


@pytest.mark.parametrize("lam", [1.0, 3.0, 6.0, 12.0, 25.6])
@pytest.mark.parametrize("delta", [0.0, 1.0, -2.0, 3.0, 6.0])
def test_cov_closed_form_matches_quadrature_of_definition(delta, lam):
    # Sec. 2.4 (b): C = (1/(Dm Dn)) int int K dV dV, computed by brute-force
    # Gauss-Legendre quadrature of the SE kernel (eq. SE) over the two cells
    x, w = _gl(60)
    S, T = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    direct = np.sum(W * np.exp(-((delta + T - S) ** 2) / (2.0 * lam * lam)))
    assert abs(O.cov_1d(delta, lam) - direct) <= 1e-13 * abs(direct)


@pytest.mark.parametrize("lam", [1.0, 6.0, 12.0, 25.6])
@pytest.mark.parametrize("delta", [0.5, -0.5, 1.5, 0.2886751345948129, 2.7113248654051871])
def test_pred_closed_form_matches_quadrature_of_definition(delta, lam):
    # Sec. 2.4 (c): t*_m = (1/Dm) int K(x*, x) dV over cell m
    x, w = _gl(60)
    direct = np.sum(w * np.exp(-((delta - x) ** 2) / (2.0 * lam * lam)))
    assert abs(O.pred_1d(delta, lam) - direct) <= 1e-13 * abs(direct)


def test_r1_flat_limit_is_poly3():
    # Sec. 2.6 / App. C: in the flat limit ell/Delta -> inf the normalised GP-R1
    # prediction vectors tend to the Poly3 Riemann-state weights
    gold = _gold("poly3_face_weights.json")
    prev = None
    for lam in (250.0, 1000.0):
        z = O.gp_weights(2, 1, lam, lam)
        err = max(np.abs(z[0, 0] - gold["east_g1"]).max(), np.abs(z[0, 1] - gold["east_g2"]).max())
        assert err < 5e-6 if lam == 1000.0 else err < 1e-4
        if prev is not None:
            assert err < prev  # converging
        prev = err


def _brute_force_weights(R, lam, dps=50):
    """Dense LU at 50 digits on C and t* assembled by mpmath quadrature of the
    kernel definitions (Sec. 2.4 (b),(c)), normalised by the sum."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    lam = mp.mpf(lam)
    cache_c, cache_t = {}, {}

    def c1(d):
        if d not in cache_c:
            f = lambda s, t: mp.exp(-((d + t - s) ** 2) / (2 * lam * lam))
            h = mp.mpf(1) / 2
            cache_c[d] = mp.quad(f, [-h, h], [-h, h])
        return cache_c[d]

    def t1(d):
        key = mp.nstr(d, 40)
        if key not in cache_t:
            h = mp.mpf(1) / 2
            cache_t[key] = mp.quad(lambda s: mp.exp(-((d - s) ** 2) / (2 * lam * lam)), [-h, h])
        return cache_t[key]

    off = O.stencil(2, R)
    n = len(off)
    Cm = mp.matrix(n, n)
    for m in range(n):
        for k in range(n):
            Cm[m, k] = c1(int(off[k][0] - off[m][0])) * c1(int(off[k][1] - off[m][1]))
    q = R + 1
    # Gauss points on [-1/2,1/2] in high precision
    xs, _ = np.polynomial.legendre.leggauss(q)
    gq = [mp.mpf(1) / 2 * mp.findroot(lambda x: mp.legendre(q, x), mp.mpf(float(x0))) for x0 in xs]
    gq = sorted(gq, reverse=True)
    out = np.zeros((4, q, n))
    for f in range(4):
        for gi, g in enumerate(gq):
            xs_, ys_ = [(mp.mpf(1) / 2, g), (-mp.mpf(1) / 2, g), (g, mp.mpf(1) / 2), (g, -mp.mpf(1) / 2)][f]
            t = mp.matrix([t1(xs_ - int(off[m][0])) * t1(ys_ - int(off[m][1])) for m in range(n)])
            z = mp.lu_solve(Cm, t)
            s = sum(z)
            out[f, gi] = [float(z[m] / s) for m in range(n)]
    return out


@pytest.mark.parametrize("R,lam", [(1, 6.0), (1, 12.0), (2, 6.0), (2, 12.0), (3, 6.0)])
def test_weights_match_brute_force_dense_solve(R, lam):
    ref = _brute_force_weights(R, lam)
    z = O.gp_weights(2, R, lam, lam)
    assert np.abs(z - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


@pytest.mark.slow
def test_r3_weights_at_flat_scale_match_brute_force():
    # the isentropic-vortex scale ell/Delta = 25.6, cond(C) ~ 4e19
    ref = _brute_force_weights(3, 25.6, dps=60)
    z = O.gp_weights(2, 3, 25.6, 25.6)
    assert np.abs(z - ref).max() <= 1e-13


@pytest.mark.parametrize("R", [1, 2, 3])
def test_weight_symmetries(R):
    off = O.stencil(2, R)
    idx = {tuple(p): k for k, p in enumerate(off)}
    z = O.gp_weights(2, R, 12.0, 12.0)
    q = z.shape[1]
    perm_mx = [idx[(-a, b)] for a, b in off]   # x mirror
    perm_my = [idx[(a, -b)] for a, b in off]   # y mirror
    perm_tr = [idx[(b, a)] for a, b in off]    # transpose
    for gi in range(q):
        gm = q - 1 - gi  # the Gauss point at -g
        np.testing.assert_allclose(z[1, gi], z[0, gi][perm_mx], atol=1e-13)   # W = mirror of E
        np.testing.assert_allclose(z[0, gm], z[0, gi][perm_my], atol=1e-13)   # -g = y-mirror
        np.testing.assert_allclose(z[2, gi], z[0, gi][perm_tr], atol=1e-13)   # N = transpose of E
        np.testing.assert_allclose(z[3, gi], z[2, gi][perm_my], atol=1e-13)   # S = mirror of N


@pytest.mark.parametrize("R", [1, 2, 3])
def test_normalisation_makes_weights_sum_to_one(R):
    # eq. normalized_z with the reading z <- z / sum(z): z^T 1 = 1
    z = O.gp_weights(2, R, 12.0, 12.0)
    np.testing.assert_allclose(z.sum(axis=2), 1.0, atol=2e-15)
    raw = O.gp_weights(2, R, 12.0, 12.0, raw=True)
    # before normalising the GP prediction already interpolates constants
    # to within a few 1e-4, so dividing by the signed sum is a small correction
    assert np.abs(raw.sum(axis=2) - 1.0).max() < 1e-3
    # the literal L1 norm would shrink every state by sum|z| > 1.6
    assert (np.abs(raw).sum(axis=2) > 1.6).all()


def test_second_derivative_weights_flat_limit_and_symmetry():
    # App. B: GP second derivative at the cell centre; flat limit -> (1,-2,1)/dx^2
    for dx in (1.0, 0.1):
        wxx, wyy = O.d2_weights(2, 1000.0 * dx, dx, dx)
        off = O.stencil(2, 1)
        target = {(0, 0): -2.0, (-1, 0): 1.0, (1, 0): 1.0, (0, 1): 0.0, (0, -1): 0.0}
        for k, (a, b) in enumerate(off):
            assert abs(wxx[k] * dx * dx - target[(a, b)]) < 2e-5
            assert abs(wyy[k] * dx * dx - target[(b, a)]) < 2e-5
    # exact on cell averages of x^2 in the flat limit: d2/dx2 = 2
    dx = 0.1
    wxx, _ = O.d2_weights(2, 1000.0 * dx, dx, dx)
    off = O.stencil(2, 1)
    avg = [((a * dx) ** 2 + dx * dx / 12.0) for a, b in off]
    assert abs(np.dot(wxx, avg) - 2.0) < 1e-4


def test_one_dimensional_weights():
    # dim = 1: the kernel product runs over x only; stencil i-R..i+R
    z = O.gp_weights(1, 2, 12.0, 12.0)
    assert z.shape == (2, 1, 5)
    np.testing.assert_allclose(z.sum(axis=2), 1.0, atol=2e-15)
    # flat limit -> the 5th-order polynomial reconstruction (2,-13,47,27,-3)/60
    z = O.gp_weights(1, 2, 400.0, 400.0)
    off = O.stencil(1, 2)[:, 0]
    ref = {-2: 2 / 60, -1: -13 / 60, 0: 47 / 60, 1: 27 / 60, 2: -3 / 60}
    for k, a in enumerate(off):
        assert abs(z[0, 0, k] - ref[a]) < 1e-4
