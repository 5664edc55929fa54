"""Seeded synthetic problem set-ups for the GP-MOOD hot path.

This module holds problem definitions only -- domains, boundary kinds, initial
conditions turned into cell averages -- and none of the method's arithmetic
(no GP weights, no fluxes, no detection).  Both the CUDA path's harness and the
CPU oracle's tests read their inputs from here.

Initial cell averages are taken with a 5x5 Gauss-Legendre rule of the
pointwise conservative variables in every cell, the conversion the paper uses
for the isentropic vortex (Sec. 5.1, a)); the same rule is used for every
problem, discontinuous ones included, so that every consumer sees the same
numbers.

Problems (sizes are arguments; the defaults are the paper-shaped workloads):
  sod_1d          Sod shock tube, 1D
  vortex          isentropic vortex (Sec. 5.1, eqs. vortex_IC_*) on a square
  density_wave    smooth density wave, an exact translation
  dmr             Mach-10 double Mach reflection (Sec. 5.2.3)
  shu_osher       Shu-Osher shock tube, 1D (Sec. 5.2.1)
  mach_jet, double_mach_jet   the Mach 100 and Mach 800 jets (Sec. 5.3)
  quadrants       four-quadrant Riemann problem with seeded random states
  shear_layer     smooth periodic double shear layer with a seeded random field
"""
from __future__ import annotations

import math

import numpy as np

BC_KINDS = ("periodic", "outflow", "reflect", "dirichlet", "dmr_bottom", "dmr_top")


def gl5():
    """5-point Gauss-Legendre nodes and weights on [-1/2, 1/2] (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(5)
    return 0.5 * x, 0.5 * w


def prim_to_cons(rho, u, v, p, gamma):
    return np.stack(
        [rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=0
    )


def cell_average(prim_fn, nx, ny, x0, x1, y0, y1, gamma, dim=2):
    """Cell averages (4, ny, nx) of the conservative variables of the pointwise
    primitive field prim_fn(x, y) -> (rho, u, v, p), by 5x5 Gauss-Legendre
    (5 points in 1D)."""
    dx = (x1 - x0) / nx
    dy = (y1 - y0) / ny
    g, w = gl5()
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    out = np.zeros((4, ny, nx))
    gy_list = [(0.0, 1.0)] if dim == 1 else list(zip(g, w))
    for gx, wx in zip(g, w):
        for gy, wy in gy_list:
            X, Y = np.meshgrid(xc + gx * dx, yc + gy * dy, indexing="xy")
            rho, u, v, p = prim_fn(X, Y)
            out += wx * wy * prim_to_cons(rho, u, v, p, gamma)
    return out


def _problem(**kw):
    base = dict(
        dim=2,
        gamma=1.4,
        bc_prim=[[1.0, 0.0, 0.0, 1.0]] * 4,
        sigma_v=5.0,
        sigma_p=5.0,
        csd_on=1,
        max_iters=0,  # 0: the implementation's own safety cap
        cfl=0.8,
        dmr_post=[1.0, 0.0, 0.0, 1.0],
        dmr_pre=[1.0, 0.0, 0.0, 1.0],
        dmr_wall_x0=0.0,
        dmr_xs0=0.0,
        dmr_xs_speed=0.0,
    )
    base.update(kw)
    return base


def sod_1d(n=128, R=2, ell_cells=12.0, cascade=None):
    """Sod tube on [0,1]: (1,0,1) | (0.125,0,0.1) at x = 0.5, outflow ends."""
    gamma = 1.4

    def prim(x, y):
        left = x < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        z = np.zeros_like(x)
        return rho, z, z, p

    dx = 1.0 / n
    U = cell_average(prim, n, 1, 0.0, 1.0, 0.0, dx, gamma, dim=1)
    return _problem(
        name=f"sod1d_{n}",
        dim=1, nx=n, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=dx,
        bc=["outflow"] * 4,
        cascade=cascade or _default_cascade(R),
        ell=ell_cells * dx, t_end=0.2, U0=U,
    )


def sod_2d(nx=64, ny=8, R=2, ell_cells=12.0, cascade=None, axis=0):
    """Sod tube along x (axis=0) or y (axis=1) on a 2D grid, outflow sides."""
    gamma = 1.4

    def prim(x, y):
        s = x if axis == 0 else y
        left = s < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        z = np.zeros_like(x)
        return rho, z, z, p

    x1 = 1.0 if axis == 0 else nx / ny
    y1 = ny / nx if axis == 0 else 1.0
    U = cell_average(prim, nx, ny, 0.0, x1, 0.0, y1, gamma)
    dx = x1 / nx
    return _problem(
        name=f"sod2d_{nx}x{ny}", nx=nx, ny=ny, x0=0.0, x1=x1, y0=0.0, y1=y1,
        bc=["outflow"] * 4, cascade=cascade or _default_cascade(R),
        ell=ell_cells * dx, t_end=0.2, U0=U,
    )


def _default_cascade(R):
    return list(range(R, -1, -1))  # e.g. R3 -> [3, 2, 1, 0]


def vortex_prim(x, y, xc, yc, beta, gamma, L):
    """Isentropic vortex (eqs. vortex_IC_dens .. vortex_IC_pres), nearest periodic image."""
    dxp = (x - xc + 0.5 * L) % L - 0.5 * L
    dyp = (y - yc + 0.5 * L) % L - 0.5 * L
    r2 = dxp * dxp + dyp * dyp
    rho = (1.0 - (gamma - 1.0) * beta**2 / (8.0 * gamma * math.pi**2) * np.exp(1.0 - r2)) ** (
        1.0 / (gamma - 1.0)
    )
    u = 1.0 - beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2)) * dyp
    v = 1.0 + beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2)) * dxp
    p = rho**gamma
    return rho, u, v, p


def vortex(n=512, lo=-5.0, hi=5.0, beta=5.0, R=3, ell=None, cascade=None, t=0.0):
    """Isentropic vortex on the periodic square [lo,hi]^2, centre at the middle,
    mean flow (1,1).  The exact solution at time t is the initial field moved by
    (t, t); t selects it.  Default ell = (hi-lo)/20, the paper's ell/L."""
    gamma = 1.4
    L = hi - lo
    c0 = 0.5 * (lo + hi)
    ell = L / 20.0 if ell is None else ell

    def prim(x, y):
        return vortex_prim(x, y, c0 + t, c0 + t, beta, gamma, L)

    U = cell_average(prim, n, n, lo, hi, lo, hi, gamma)
    return _problem(
        name=f"vortex_{n}", nx=n, ny=n, x0=lo, x1=hi, y0=lo, y1=hi,
        bc=["periodic"] * 4, cascade=cascade or _default_cascade(R),
        ell=ell, t_end=L, U0=U,
    )


def density_wave(n=32, amp=0.2, R=1, ell=0.2, cascade=None, t=0.0, nx=None, ny=None,
                 kx=1, ky=1):
    """rho = 1 + amp sin(2 pi (kx x + ky y - (kx+ky) t)), u = v = 1, p = 1 on the
    periodic unit square: an exact translation with velocity (1,1)."""
    gamma = 1.4
    nx = nx or n
    ny = ny or n

    def prim(x, y):
        rho = 1.0 + amp * np.sin(2.0 * math.pi * (kx * (x - t) + ky * (y - t)))
        one = np.ones_like(x)
        return rho, one, one, one

    U = cell_average(prim, nx, ny, 0.0, 1.0, 0.0, 1.0, gamma)
    return _problem(
        name=f"wave_{nx}x{ny}", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
        bc=["periodic"] * 4, cascade=cascade or _default_cascade(R),
        ell=ell, t_end=1.0, U0=U,
    )


def dmr(nx=4096, ny=1024, R=3, ell_cells=12.0, cascade=None):
    """Mach-10 shock at 60 degrees to a reflecting wall starting at x = 1/6 on
    [0,4] x [0,1].  Pre-shock (1.4, 0, 0, 1); post-shock (8, 8.25 cos 30,
    -8.25 sin 30, 116.5).  Left: post-shock inflow; right: outflow; bottom:
    post-shock for x < 1/6, reflecting beyond; top: the exact shock position
    x_s(t) = 1/6 + (1 + 20 t)/sqrt(3)."""
    gamma = 1.4
    post = [8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5]
    pre = [1.4, 0.0, 0.0, 1.0]
    x_wall = 1.0 / 6.0

    def prim(x, y):
        behind = x < x_wall + y / math.tan(math.pi / 3)
        out = [np.where(behind, a, b) for a, b in zip(post, pre)]
        return out[0], out[1], out[2], out[3]

    U = cell_average(prim, nx, ny, 0.0, 4.0, 0.0, 1.0, gamma)
    dx = 4.0 / nx
    return _problem(
        name=f"dmr_{nx}x{ny}", nx=nx, ny=ny, x0=0.0, x1=4.0, y0=0.0, y1=1.0,
        bc=["dirichlet", "outflow", "dmr_bottom", "dmr_top"],
        bc_prim=[post, pre, post, post],
        dmr_post=post, dmr_pre=pre, dmr_wall_x0=x_wall,
        dmr_xs0=x_wall + 1.0 / math.sqrt(3.0), dmr_xs_speed=20.0 / math.sqrt(3.0),
        cascade=cascade or _default_cascade(R), ell=ell_cells * dx, t_end=0.2, U0=U,
    )


def mach_jet(n=600, R=3, ell_cells=12.0, cascade=None):
    """Single Mach 100 light jet (Sec. 5.3): the outflow box [0,1.5]^2 with the
    jet (gamma, 0, 100, 1) entering through the slit 0.7 <= x <= 0.8 at y = 0
    into the ambient (10 gamma, 0, 0, 1); HLL; t_end 0.04.  The paper's
    cascades are GP-MOOD3/5/7: [1, 0], [2, 1, 0], [3, 1, 0]."""
    gamma = 1.4
    jet = [gamma, 0.0, 100.0, 1.0]

    def prim(x, y):
        one = np.ones_like(x)
        return 10.0 * gamma * one, 0.0 * one, 0.0 * one, one

    U = cell_average(prim, n, n, 0.0, 1.5, 0.0, 1.5, gamma)
    dx = 1.5 / n
    return _problem(
        name=f"machjet_{n}", nx=n, ny=n, x0=0.0, x1=1.5, y0=0.0, y1=1.5,
        bc=["outflow", "outflow", "jet", "outflow"], jet_x=(0.7, 0.8), jet_prim=[jet, jet],
        riemann="hll", cascade=cascade or ([R, 1, 0] if R > 1 else [1, 0]),
        ell=ell_cells * dx, t_end=0.04, U0=U,
    )


def double_mach_jet(n=600, R=3, ell_cells=12.0, cascade=None):
    """Double Mach 800 jet collision (Sec. 5.3): the single-jet box with the
    ambient density stratified as rho = -9.24 y + 14 (u = v = 0, p = 1) and
    jets (gamma, 0, +-800, 1) through 0.7 <= x <= 0.8 at y = 0 and y = 1.5.
    The printed jet velocity is +800 at both ends; the top jet is injected
    into the domain, so it enters with v = -800.  HLL; t_end 0.005."""
    gamma = 1.4

    def prim(x, y):
        one = np.ones_like(x)
        return -9.24 * y + 14.0, 0.0 * one, 0.0 * one, one

    U = cell_average(prim, n, n, 0.0, 1.5, 0.0, 1.5, gamma)
    dx = 1.5 / n
    return _problem(
        name=f"doublejet_{n}", nx=n, ny=n, x0=0.0, x1=1.5, y0=0.0, y1=1.5,
        bc=["outflow", "outflow", "jet", "jet"], jet_x=(0.7, 0.8),
        jet_prim=[[gamma, 0.0, 800.0, 1.0], [gamma, 0.0, -800.0, 1.0]],
        riemann="hll", cascade=cascade or ([R, 1, 0] if R > 1 else [1, 0]),
        ell=ell_cells * dx, t_end=0.005, U0=U,
    )


# The paper's four schemes (Sec. 3.1): cascade, reconstruction and time
# integrator.  GP-MOOD5/7 step with SSP-RK4 and a time step reduced by
# Delta^((2R+1)/4 - 1) (Sec. 5.1 b); GP-MOOD3 and POL-MOOD3 with SSP-RK3.
SCHEMES = {
    "GP-MOOD3": dict(cascade=[1, 0], recon="gp", rk=3),
    "GP-MOOD5": dict(cascade=[2, 1, 0], recon="gp", rk=4),
    "GP-MOOD7": dict(cascade=[3, 1, 0], recon="gp", rk=4),
    "POL-MOOD3": dict(cascade=[1, 0], recon="poly3", rk=3),
}


def scheme_cfl(name, delta, cfl=0.8, reduce=True):
    """CFL number of a scheme: cfl, times Delta^((2R+1)/4 - 1) for the
    SSP-RK4 schemes when reduce is set."""
    sch = SCHEMES[name]
    if sch["rk"] != 4 or not reduce:
        return cfl
    R = sch["cascade"][0]
    return cfl * delta ** ((2 * R + 1) / 4.0 - 1.0)


def shu_osher(n=256, scheme="GP-MOOD7", ell_cells=6.0, csd_on=1, reduce_dt=True):
    """Shu-Osher shock tube (Sec. 5.2.1) on [0, 9], 1D: a Mach 3 shock at
    x = 0.5, (rho, u, p) = (3.857143, 2.629369, 10.33333) behind it, and
    (1 + 0.2 sin(5 (x - 4.5)), 0, 1) ahead; t_end 1.8, ell = 6 Delta.  The
    left end holds the post-shock state (fixed inflow).  The right end is
    zero-gradient: ahead of the shock the gas is at rest at uniform pressure,
    a state whose face fluxes do not depend on the density, and the shock
    stays short of x = 9 up to t_end, so this equals holding the initial
    values there."""
    gamma = 1.4
    left = [3.857143, 2.629369, 0.0, 10.33333]

    def prim(x, y):
        behind = x < 0.5
        rho = np.where(behind, left[0], 1.0 + 0.2 * np.sin(5.0 * (x - 4.5)))
        u = np.where(behind, left[1], 0.0)
        p = np.where(behind, left[3], 1.0)
        return rho, u, np.zeros_like(x), p

    dx = 9.0 / n
    U = cell_average(prim, n, 1, 0.0, 9.0, 0.0, dx, gamma, dim=1)
    sch = SCHEMES[scheme]
    return _problem(
        name=f"shuosher_{n}_{scheme}", dim=1, nx=n, ny=1, x0=0.0, x1=9.0, y0=0.0, y1=dx,
        bc=["dirichlet", "outflow", "outflow", "outflow"],
        bc_prim=[left, [1.0, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 1.0]],
        cascade=list(sch["cascade"]), recon=sch["recon"], rk=sch["rk"],
        cfl=scheme_cfl(scheme, dx, reduce=reduce_dt), csd_on=csd_on,
        ell=ell_cells * dx, t_end=1.8, U0=U,
    )


def quadrant_states(seed=0, count=1):
    """count draws of four quadrant states (rho, u, v, p) with rho in [0.1,2],
    p in [0.05,2], u,v in [-1,1] from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    states = np.empty((count, 4, 4))
    for k in range(count):
        for q in range(4):
            states[k, q] = [rng.uniform(0.1, 2.0), rng.uniform(-1.0, 1.0),
                            rng.uniform(-1.0, 1.0), rng.uniform(0.05, 2.0)]
    return states


def quadrants(n=256, R=3, ell_cells=12.0, cascade=None, seed=0, states=None, ny=None):
    """Four-quadrant Riemann problem on [0,1]^2 split at (1/2, 1/2), outflow
    sides.  Quadrant order: (x>1/2,y>1/2), (x<1/2,y>1/2), (x<1/2,y<1/2),
    (x>1/2,y<1/2)."""
    gamma = 1.4
    ny = ny or n
    st = quadrant_states(seed)[0] if states is None else np.asarray(states)

    def prim(x, y):
        q = np.where(y > 0.5, np.where(x > 0.5, 0, 1), np.where(x < 0.5, 2, 3))
        return tuple(st[q, k] for k in range(4))

    U = cell_average(prim, n, ny, 0.0, 1.0, 0.0, 1.0, gamma)
    dx = 1.0 / n
    return _problem(
        name=f"quad_{n}x{ny}", nx=n, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
        bc=["outflow"] * 4, cascade=cascade or _default_cascade(R),
        ell=min(ell_cells * dx, ell_cells / ny), t_end=0.25, U0=U,
    )


def gaussian_random_field(n, corr=0.05, rms=1e-2, seed=0):
    """Periodic random field on an n x n grid: white noise filtered by a
    Gaussian spectrum of correlation length corr, scaled to the given RMS."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    filt = np.exp(-0.5 * (2.0 * math.pi * corr) ** 2 * (KX**2 + KY**2))
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    f -= f.mean()
    return f * (rms / np.sqrt(np.mean(f * f)))


def shear_layer(n=1024, R=2, ell_cells=12.0, cascade=None, seed=0, width=0.05, u0=0.5,
                p0=2.5, ub=0.3, vb=0.2):
    """Periodic double shear layer on [0,1]^2: rho = 1 + 0.1 * prof(y),
    u = ub + u0 * prof(y), v = vb, p = p0, with prof = (tanh((y-1/4)/w) -
    tanh((y-3/4)/w))/2, plus a seeded Gaussian random field (RMS 1e-2,
    correlation 0.05) added to the density cell averages.  The uniform
    background flow (ub, vb) keeps the contact speed of every face away from
    zero, where the HLLC flux is not differentiable."""
    gamma = 1.4

    def prof(y):
        return 0.5 * (np.tanh((y - 0.25) / width) - np.tanh((y - 0.75) / width))

    def prim(x, y):
        pr = prof(y)
        return (1.0 + 0.1 * pr, ub + u0 * pr, vb * np.ones_like(x), p0 * np.ones_like(x))

    U = cell_average(prim, n, n, 0.0, 1.0, 0.0, 1.0, gamma)
    drho = gaussian_random_field(n, seed=seed)
    # add the perturbation to rho while keeping velocity and pressure
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    rho2 = rho + drho
    U = prim_to_cons(rho2, u, v, p, gamma)
    dx = 1.0 / n
    return _problem(
        name=f"shear_{n}", nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
        bc=["periodic"] * 4, cascade=cascade or _default_cascade(R),
        ell=ell_cells * dx, t_end=None, U0=U,
    )


def uniform(nx=16, ny=16, R=3, state=(1.0, 0.3, -0.2, 1.0), bc="periodic", ell=0.2):
    gamma = 1.4

    def prim(x, y):
        return tuple(np.full_like(x, s) for s in state)

    U = cell_average(prim, nx, ny, 0.0, 1.0, 0.0, 1.0, gamma)
    return _problem(
        name=f"uniform_{nx}x{ny}", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
        bc=[bc] * 4, cascade=_default_cascade(R), ell=ell, t_end=None, U0=U,
    )


def quadrant_batch(count=64, sizes=(128, 256, 512, 1024), seed=0, R=3, ell_cells=12.0):
    """count four-quadrant problems on [0,1]^2: the grid size of each drawn
    uniformly from `sizes` and its quadrant states from quadrant_states,
    both with numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    states = quadrant_states(seed=seed + 1, count=count)
    return [quadrants(n=int(n), R=R, ell_cells=ell_cells, states=states[k]) for k, n in enumerate(ns)]
