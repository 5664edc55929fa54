"""ctypes binding of the plain FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gpmood_oracle.c")
LIB = os.path.join(HERE, "_build", "libgpmood_oracle.so")

BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3, "dmr_bottom": 4, "dmr_top": 5,
      "jet": 6}
RIEMANN = {"hllc": 0, "hll": 1}
RECON = {"gp": 0, "poly3": 1}
ACCEPT_CSD, ACCEPT_PLATEAU, ACCEPT_DMP, ACCEPT_U2 = 1, 2, 3, 4
FAIL_CAD, FAIL_PAD, FAIL_U2 = -1, -2, -3


# no fast-math, no FMA contraction
CFLAGS = ("gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off")


def build(force=False):
    """Compile the oracle with gcc (CFLAGS)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([*CFLAGS, "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


class Config(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("bc", C.c_int * 4), ("bc_prim", (C.c_double * 4) * 4), ("gamma", C.c_double),
        ("ncascade", C.c_int), ("cascade", C.c_int * 4), ("ell", C.c_double),
        ("sigma_v", C.c_double), ("sigma_p", C.c_double), ("csd_on", C.c_int),
        ("max_iters", C.c_int),
        ("dmr_post", C.c_double * 4), ("dmr_pre", C.c_double * 4),
        ("dmr_wall_x0", C.c_double), ("dmr_xs0", C.c_double), ("dmr_xs_speed", C.c_double),
        ("rk", C.c_int), ("riemann", C.c_int), ("jet_x0", C.c_double), ("jet_x1", C.c_double),
        ("jet_prim", (C.c_double * 4) * 2), ("poly3", C.c_int),
    ]


class StepStats(C.Structure):
    _fields_ = [("dt", C.c_double), ("iters", C.c_int * 5), ("nbad_first", C.c_int * 5),
                ("nbad_total", C.c_int * 5), ("status", C.c_int)]


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = C.CDLL(build())
        d, i, p = C.c_double, C.c_int, C.c_void_p
        L.orc_create.argtypes = [C.POINTER(Config), C.POINTER(p)]
        L.orc_destroy.argtypes = [p]
        L.orc_destroy.restype = None
        L.orc_ghost_width.argtypes = [p]
        L.orc_stencil.argtypes = [i, i, p]
        L.orc_gauss_rule.argtypes = [i, p, p]
        L.orc_pred_1d.argtypes = [d, d]
        L.orc_pred_1d.restype = d
        L.orc_cov_1d.argtypes = [d, d]
        L.orc_cov_1d.restype = d
        L.orc_gp_weights.argtypes = [i, i, d, d, p, p, p]
        L.orc_gp_weights_raw.argtypes = [i, i, d, d, p]
        L.orc_d2_weights.argtypes = [i, d, d, d, p, p]
        L.orc_residual.argtypes = [p, p, p, d, p]
        L.orc_residual_cad.argtypes = [p, p, p, d, p, p]
        L.orc_dt.argtypes = [p, p, d]
        L.orc_dt.restype = d
        L.orc_step.argtypes = [p, p, d, d, d, p, p, C.POINTER(StepStats)]
        L.orc_stage.argtypes = [p, p, d, d, p, p, p, p, p]
        L.orc_detect_cell.argtypes = [p, p, i, i, p]
        L.orc_fill_ghosts.argtypes = [p, p, d, p]
        L.orc_hllc.argtypes = [p, p, d, i, p]
        L.orc_hllc.restype = None
        L.orc_hll.argtypes = [p, p, d, i, p]
        L.orc_hll.restype = None
        L.orc_curvature.argtypes = [p, p, i, i, i]
        L.orc_curvature.restype = d
        L.orc_poly3_eval.argtypes = [i, p, d, d]
        L.orc_poly3_eval.restype = d
        _lib_handle = L
    return _lib_handle


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def stencil(dim, R):
    off = np.zeros(2 * 25, dtype=np.int32)
    n = lib().orc_stencil(dim, R, _ptr(off))
    return off[: 2 * n].reshape(n, 2)


def gauss_rule(q):
    g = np.zeros(4)
    w = np.zeros(4)
    if lib().orc_gauss_rule(q, _ptr(g), _ptr(w)) != q:
        raise ValueError(q)
    return g[:q], w[:q]


def pred_1d(delta, lam):
    return lib().orc_pred_1d(float(delta), float(lam))


def cov_1d(delta, lam):
    return lib().orc_cov_1d(float(delta), float(lam))


def gp_weights(dim, R, lamx, lamy, raw=False):
    """z[face][g][m], faces (E, W, N, S) (dim 1: E, W)."""
    z = np.zeros(4 * 4 * 25)
    nq = C.c_int(0)
    nn = C.c_int(0)
    rc = lib().orc_gp_weights(dim, R, lamx, lamy, _ptr(z), C.byref(nq), C.byref(nn))
    if rc != 0:
        raise RuntimeError(f"orc_gp_weights rc={rc}")
    q, n = nq.value, nn.value
    nf = 4 if dim == 2 else 2
    if raw:
        z = np.zeros(4 * 4 * 25)
        lib().orc_gp_weights_raw(dim, R, lamx, lamy, _ptr(z))
    return z[: nf * q * n].reshape(nf, q, n)


def d2_weights(dim, ell, dx, dy):
    wxx = np.zeros(25)
    wyy = np.zeros(25)
    n = lib().orc_d2_weights(dim, ell, dx, dy, _ptr(wxx), _ptr(wyy))
    if n < 0:
        raise RuntimeError("orc_d2_weights")
    return wxx[:n], wyy[:n]


def poly3_eval(dim, qv, xs, ys):
    """Poly3 (eq. poly3, App. C) of the R = 1 stencil values qv (orc_stencil
    order) at (xs, ys) in cell units from the cell centre."""
    qv = np.ascontiguousarray(qv, dtype=np.float64)
    return lib().orc_poly3_eval(int(dim), _ptr(qv), float(xs), float(ys))


def hllc(UL, UR, gamma=1.4, direction=0):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(4)
    lib().orc_hllc(_ptr(UL), _ptr(UR), gamma, direction, _ptr(F))
    return F


def hll(UL, UR, gamma=1.4, direction=0):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(4)
    lib().orc_hll(_ptr(UL), _ptr(UR), gamma, direction, _ptr(F))
    return F


def make_config(prob):
    cfg = Config()
    cfg.dim = int(prob.get("dim", 2))
    cfg.nx, cfg.ny = int(prob["nx"]), int(prob["ny"])
    cfg.x0, cfg.x1, cfg.y0, cfg.y1 = prob["x0"], prob["x1"], prob["y0"], prob["y1"]
    for s in range(4):
        cfg.bc[s] = BC[prob["bc"][s]]
        for k in range(4):
            cfg.bc_prim[s][k] = prob["bc_prim"][s][k]
    cfg.gamma = prob["gamma"]
    cas = list(prob["cascade"])
    cfg.ncascade = len(cas)
    for k, r in enumerate(cas):
        cfg.cascade[k] = r
    cfg.ell = prob["ell"]
    cfg.sigma_v, cfg.sigma_p = prob["sigma_v"], prob["sigma_p"]
    cfg.csd_on = int(prob["csd_on"])
    cfg.max_iters = int(prob.get("max_iters", 0)) or 1000000
    for k in range(4):
        cfg.dmr_post[k] = prob["dmr_post"][k]
        cfg.dmr_pre[k] = prob["dmr_pre"][k]
    cfg.dmr_wall_x0 = prob["dmr_wall_x0"]
    cfg.dmr_xs0 = prob["dmr_xs0"]
    cfg.dmr_xs_speed = prob["dmr_xs_speed"]
    cfg.rk = int(prob.get("rk", 3))
    cfg.riemann = RIEMANN[prob.get("riemann", "hllc")]
    cfg.jet_x0, cfg.jet_x1 = prob.get("jet_x", (0.0, 0.0))
    for side, P in enumerate(prob.get("jet_prim", ([1.0, 0.0, 0.0, 1.0],) * 2)):
        for k in range(4):
            cfg.jet_prim[side][k] = P[k]
    cfg.poly3 = RECON[prob.get("recon", "gp")]
    return cfg


class Oracle:
    """One problem configuration with its precomputed weights."""

    def __init__(self, prob):
        self.prob = prob
        self.cfg = make_config(prob)
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.cfg), C.byref(h))
        if rc != 0:
            raise RuntimeError(f"orc_create failed rc={rc}")
        self.h = h
        self.nx, self.ny = self.cfg.nx, self.cfg.ny
        self.H = lib().orc_ghost_width(self.h)

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (4, self.ny, self.nx), U.shape
        return U

    def fill_ghosts(self, U, t=0.0):
        U = self._state(U)
        Xg = np.zeros((4, self.ny + 2 * self.H, self.nx + 2 * self.H))
        lib().orc_fill_ghosts(self.h, _ptr(U), t, _ptr(Xg))
        return Xg

    def residual(self, U, ord_map, t=0.0, want_cad=False):
        """F_nabla at the radii ord_map; with want_cad also the per-cell
        face-state check at those radii (1: a state of the cell failed)."""
        U = self._state(U)
        o = np.ascontiguousarray(ord_map, dtype=np.uint8)
        Fn = np.zeros_like(U)
        cad = np.zeros((self.ny, self.nx), dtype=np.uint8)
        rc = lib().orc_residual_cad(self.h, _ptr(U), _ptr(o), t, _ptr(Fn), _ptr(cad))
        if rc != 0:
            raise RuntimeError(rc)
        return (Fn, cad) if want_cad else Fn

    def dt(self, U, cfl):
        return lib().orc_dt(self.h, _ptr(self._state(U)), cfl)

    @property
    def nstages(self):
        return 5 if self.cfg.rk == 4 else 3

    def step(self, U, t=0.0, cfl=None, dt_fixed=0.0):
        """One SSP-RK3 (or SSP-RK4) step.  Returns (U_new, stats dict,
        ord[S,ny,nx], first-pass bad[S,ny,nx]), S the number of stages."""
        U = self._state(U).copy()
        cfl = self.prob["cfl"] if cfl is None else cfl
        nc = self.nx * self.ny
        S = self.nstages
        ordm = np.zeros(S * nc, dtype=np.uint8)
        bad = np.zeros(S * nc, dtype=np.uint8)
        st = StepStats()
        rc = lib().orc_step(self.h, _ptr(U), t, cfl, dt_fixed, _ptr(ordm), _ptr(bad), C.byref(st))
        if rc != 0:
            raise RuntimeError(f"orc_step rc={rc}")
        stats = dict(dt=st.dt, iters=list(st.iters)[:S], nbad_first=list(st.nbad_first)[:S],
                     nbad_total=list(st.nbad_total)[:S])
        return U, stats, ordm.reshape(S, self.ny, self.nx), bad.reshape(S, self.ny, self.nx)

    def stage(self, X, ts, dt):
        X = self._state(X)
        Y = np.zeros_like(X)
        o = np.zeros(self.nx * self.ny, dtype=np.uint8)
        b = np.zeros(self.nx * self.ny, dtype=np.uint8)
        it = C.c_int(0)
        tot = C.c_int(0)
        rc = lib().orc_stage(self.h, _ptr(X), ts, dt, _ptr(Y), _ptr(o), _ptr(b), C.byref(it),
                             C.byref(tot))
        if rc != 0:
            raise RuntimeError(f"orc_stage rc={rc}")
        return Y, o.reshape(self.ny, self.nx), b.reshape(self.ny, self.nx), it.value, tot.value

    def detect_cell(self, Xg, i, j, Y4):
        Xg = np.ascontiguousarray(Xg, dtype=np.float64)
        Y4 = np.ascontiguousarray(Y4, dtype=np.float64)
        return lib().orc_detect_cell(self.h, _ptr(Xg), i, j, _ptr(Y4))

    def curvature(self, Xg, d, i, j):
        Xg = np.ascontiguousarray(Xg, dtype=np.float64)
        return lib().orc_curvature(self.h, _ptr(Xg), d, i, j)

    def run(self, U, t_end, cfl=None, max_steps=10**9):
        """Steps to t_end with the last step clipped.  Returns (U, nsteps, t)."""
        U = self._state(U).copy()
        t = 0.0
        n = 0
        cfl = self.prob["cfl"] if cfl is None else cfl
        while t < t_end * (1 - 1e-14) and n < max_steps:
            dt = self.dt(U, cfl)
            if t + dt > t_end:
                dt = t_end - t
            U, _, _, _ = self.step(U, t, cfl, dt_fixed=dt)
            t += dt
            n += 1
        return U, n, t
