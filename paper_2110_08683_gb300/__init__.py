"""GB300-native GP-MOOD hot path: Python binding of the C ABI in include/gpmood.h.

Argument marshalling only: every step of the method runs in the CUDA library
libgpmood.so (built in-tree by ``build.build()``).  There is no CPU fallback:
loading fails loudly if the library is missing or no CUDA device is present.

Function names follow the C ABI (gpmood_create, gpmood_set_state,
gpmood_get_state, gpmood_step, gpmood_step_dt, gpmood_run, gpmood_step_async,
gpmood_sync, gpmood_launch_count, gpmood_flags, gpmood_destroy,
gpmood_strerror); ``GPMood`` wraps a handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3, "dmr_bottom": 4, "dmr_top": 5,
      "jet": 6}
RIEMANN = {"hllc": 0, "hll": 1}
RECON = {"gp": 0, "poly3": 1}  # poly3: POL-MOOD3 (Sec. 3.1 (iv)), R_max = 1
FP64, FP32 = 0, 1

E_CODES = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "device allocation failed",
           -4: "GP covariance matrix not positive definite", -5: "MOOD iteration cap reached",
           -6: "time step not positive or not finite", -7: "no state set",
           -8: "grid too large for the static scratch",
           -9: "a grid-wide barrier of the MOOD loop timed out"}


class GpmoodError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {gpmood_strerror(code)} ({code})")
        self.code = code


class Grid(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("bc", C.c_int * 4), ("bc_prim", (C.c_double * 4) * 4),
        ("dmr_post", C.c_double * 4), ("dmr_pre", C.c_double * 4),
        ("dmr_wall_x0", C.c_double), ("dmr_xs0", C.c_double), ("dmr_xs_speed", C.c_double),
        ("jet_x0", C.c_double), ("jet_x1", C.c_double), ("jet_prim", (C.c_double * 4) * 2),
        ("dim", C.c_int),
    ]


class Options(C.Structure):
    _fields_ = [
        ("ncascade", C.c_int), ("cascade", C.c_int * 4), ("precision", C.c_int),
        ("sigma_v", C.c_double), ("sigma_p", C.c_double), ("csd_off", C.c_int),
        ("max_mood_iters", C.c_int), ("riemann", C.c_int), ("rk", C.c_int),
        ("eager", C.c_int), ("recon", C.c_int), ("serial_launch", C.c_int),
        ("split_faces", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("dt", C.c_double), ("nsteps", C.c_longlong),
        ("iters", C.c_int * 5), ("nbad_first", C.c_int * 5), ("nbad_total", C.c_int * 5),
        ("nfog_pad", C.c_int * 5), ("status", C.c_int),
    ]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libgpmood.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libgpmood.so not found at {path}; run build()")
    L = C.CDLL(path)
    p, i, d = C.c_void_p, C.c_int, C.c_double
    L.gpmood_create.argtypes = [C.POINTER(Grid), d, i, d, C.POINTER(Options), C.POINTER(p)]
    L.gpmood_set_stream.argtypes = [p, p]
    L.gpmood_set_state.argtypes = [p, p, i]
    L.gpmood_get_state.argtypes = [p, p, i]
    L.gpmood_set_time.argtypes = [p, d]
    L.gpmood_step.argtypes = [p, d, C.POINTER(d)]
    L.gpmood_step_dt.argtypes = [p, d]
    L.gpmood_run.argtypes = [p, d, d, C.POINTER(C.c_longlong)]
    L.gpmood_step_async.argtypes = [p, d]
    L.gpmood_sync.argtypes = [p]
    L.gpmood_launch_count.argtypes = [p, C.POINTER(C.c_longlong)]
    L.gpmood_flags.argtypes = [p, p, p, C.POINTER(Stats)]
    L.gpmood_destroy.argtypes = [p]
    L.gpmood_strerror.argtypes = [i]
    L.gpmood_strerror.restype = C.c_char_p
    L.gpmood_last_launches.argtypes = [p]
    L.gpmood_profile.argtypes = [p, i]
    L.gpmood_step_record.argtypes = [p, d, d, p, p, C.POINTER(d)]
    L.gpmood_step_frozen.argtypes = [p, p, d]
    L.gpmood_step_adjoint.argtypes = [p, p, p, d, d, p, p]
    L.gpmood_state_tape_bytes.argtypes = [p, C.POINTER(C.c_size_t)]
    L.gpmood_step_record_states.argtypes = [p, d, d, p, p, p, C.POINTER(d)]
    L.gpmood_step_adjoint_states.argtypes = [p, p, p, p, d, d, p, p]
    L.gpmood_batch_create.argtypes = [C.POINTER(Grid), i, d, i, C.POINTER(d), C.POINTER(Options),
                                      C.POINTER(p)]
    L.gpmood_batch_set_stream.argtypes = [p, p]
    L.gpmood_batch_set_state.argtypes = [p, p, i]
    L.gpmood_batch_get_state.argtypes = [p, p, i]
    L.gpmood_batch_step.argtypes = [p, d]
    L.gpmood_batch_run.argtypes = [p, d, d, C.POINTER(C.c_longlong)]
    L.gpmood_batch_info.argtypes = [p, p, p, p, C.POINTER(Stats)]
    L.gpmood_batch_tuning.argtypes = [p, p, p]
    L.gpmood_batch_grids.argtypes = [p, p, p]
    L.gpmood_batch_profile.argtypes = [p, i]
    L.gpmood_batch_kernel_times.argtypes = [p, p, p]
    L.gpmood_batch_destroy.argtypes = [p]
    L.gpmood_step_noalloc.argtypes = [C.POINTER(Grid), d, i, d, C.POINTER(Options), p, p, d, d,
                                      C.POINTER(d), p]
    L.gpmood_kernel_times.argtypes = [p, p, p]
    _lib = L
    return L


def _check(rc, what):
    if rc != 0:
        raise GpmoodError(rc, what)


def gpmood_strerror(code):
    return E_CODES.get(code, "unknown error")


def make_grid(prob):
    g = Grid()
    g.nx, g.ny = int(prob["nx"]), int(prob["ny"])
    g.x0, g.x1, g.y0, g.y1 = prob["x0"], prob["x1"], prob["y0"], prob["y1"]
    for s in range(4):
        g.bc[s] = BC[prob["bc"][s]]
        for k in range(4):
            g.bc_prim[s][k] = prob["bc_prim"][s][k]
    for k in range(4):
        g.dmr_post[k] = prob["dmr_post"][k]
        g.dmr_pre[k] = prob["dmr_pre"][k]
    g.dmr_wall_x0 = prob["dmr_wall_x0"]
    g.dmr_xs0 = prob["dmr_xs0"]
    g.dmr_xs_speed = prob["dmr_xs_speed"]
    g.jet_x0, g.jet_x1 = prob.get("jet_x", (0.0, 0.0))
    for side, P in enumerate(prob.get("jet_prim", ([1.0, 0.0, 0.0, 1.0],) * 2)):
        for k in range(4):
            g.jet_prim[side][k] = P[k]
    g.dim = int(prob.get("dim", 2))
    return g


def make_options(prob, precision=FP64, eager=False):
    o = Options()
    cas = list(prob["cascade"])
    o.ncascade = len(cas)
    for k, r in enumerate(cas):
        o.cascade[k] = r
    o.precision = precision
    o.sigma_v, o.sigma_p = prob["sigma_v"], prob["sigma_p"]
    o.csd_off = 0 if prob["csd_on"] else 1
    o.max_mood_iters = int(prob.get("max_iters", 0))
    o.rk = int(prob.get("rk", 3))
    o.riemann = RIEMANN[prob.get("riemann", "hllc")]
    o.recon = RECON[prob.get("recon", "gp")]
    o.serial_launch = int(prob.get("serial_launch", 0))
    o.split_faces = int(prob.get("split_faces", 0))
    o.eager = 1 if eager else 0
    return o


def gpmood_create(grid, gamma, R_max, ell, opts):
    h = C.c_void_p()
    _check(load().gpmood_create(C.byref(grid), gamma, R_max, ell, C.byref(opts), C.byref(h)),
           "gpmood_create")
    return h


def _ptr_of(U):
    """(pointer, on_device) of a contiguous float64 numpy array or CUDA tensor."""
    if hasattr(U, "data_ptr") and getattr(U, "is_cuda", False):
        return C.c_void_p(U.data_ptr()), 1
    return U.ctypes.data_as(C.c_void_p), 0


def gpmood_set_state(h, U):
    p, dev = _ptr_of(U)
    _check(load().gpmood_set_state(h, p, dev), "gpmood_set_state")


def gpmood_set_time(h, t):
    _check(load().gpmood_set_time(h, t), "gpmood_set_time")


def gpmood_get_state(h, out):
    p, dev = _ptr_of(out)
    _check(load().gpmood_get_state(h, p, dev), "gpmood_get_state")
    return out


def gpmood_step(h, cfl, want_dt=False):
    if want_dt:
        dt = C.c_double(0.0)
        _check(load().gpmood_step(h, cfl, C.byref(dt)), "gpmood_step")
        return dt.value
    _check(load().gpmood_step(h, cfl, None), "gpmood_step")
    return None


def gpmood_step_dt(h, dt):
    _check(load().gpmood_step_dt(h, dt), "gpmood_step_dt")


def gpmood_run(h, t_end, cfl):
    n = C.c_longlong(0)
    _check(load().gpmood_run(h, t_end, cfl, C.byref(n)), "gpmood_run")
    return n.value


def gpmood_step_async(h, cfl):
    _check(load().gpmood_step_async(h, cfl), "gpmood_step_async")


def gpmood_sync(h):
    _check(load().gpmood_sync(h), "gpmood_sync")


def gpmood_launch_count(h):
    n = C.c_longlong(0)
    _check(load().gpmood_launch_count(h, C.byref(n)), "gpmood_launch_count")
    return n.value


def gpmood_flags(h, nx, ny, maps=True, nstages=3):
    """final radii and first-pass troubled maps [S][ny][nx] and the stats of
    the last step (S = 3 for SSP-RK3, 5 for SSP-RK4)"""
    st = Stats()
    S = nstages
    if maps:
        order = np.zeros((S, ny, nx), dtype=np.uint8)
        first = np.zeros((S, ny, nx), dtype=np.uint8)
        _check(load().gpmood_flags(h, order.ctypes.data_as(C.c_void_p),
                                   first.ctypes.data_as(C.c_void_p), C.byref(st)), "gpmood_flags")
    else:
        order = first = None
        _check(load().gpmood_flags(h, None, None, C.byref(st)), "gpmood_flags")
    stats = dict(t=st.t, dt=st.dt, nsteps=st.nsteps, iters=list(st.iters)[:S],
                 nbad_first=list(st.nbad_first)[:S], nbad_total=list(st.nbad_total)[:S],
                 nfog_pad=list(st.nfog_pad)[:S], status=st.status)
    return order, first, stats


def gpmood_destroy(h):
    if h:
        load().gpmood_destroy(h)


def gpmood_set_stream(h, stream_ptr):
    _check(load().gpmood_set_stream(h, C.c_void_p(stream_ptr)), "gpmood_set_stream")


def gpmood_last_launches(h):
    return load().gpmood_last_launches(h)


def gpmood_step_noalloc(prob, U_in_ptr, U_out_ptr, t, cfl, precision=FP64, stream_ptr=0):
    """One step through the allocation-free entry point: U_in_ptr / U_out_ptr
    are device pointers to [4][ny][nx] float64 cell averages.  Returns dt."""
    dt = C.c_double(0.0)
    cas = list(prob["cascade"])
    g, o = make_grid(prob), make_options(prob, precision)
    _check(load().gpmood_step_noalloc(C.byref(g), prob["gamma"], cas[0], prob["ell"], C.byref(o),
                                      C.c_void_p(U_in_ptr), C.c_void_p(U_out_ptr), t, cfl,
                                      C.byref(dt), C.c_void_p(stream_ptr)),
           "gpmood_step_noalloc")
    return dt.value


KERNEL_CLASSES = ("dt", "ghost", "faces_x", "faces_y", "update", "mood")


def gpmood_profile(h, enable):
    _check(load().gpmood_profile(h, 1 if enable else 0), "gpmood_profile")


def gpmood_kernel_times(h):
    ms = np.zeros(len(KERNEL_CLASSES))
    n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    _check(load().gpmood_kernel_times(h, ms.ctypes.data_as(C.c_void_p),
                                      n.ctypes.data_as(C.c_void_p)), "gpmood_kernel_times")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


class GPMood:
    """One GP-MOOD problem on the GPU: a handle of the C ABI."""

    def __init__(self, prob, precision="fp64", eager=False):
        self.prob = prob
        self.nx, self.ny = int(prob["nx"]), int(prob["ny"])
        self.precision = FP32 if precision in ("fp32", FP32) else FP64
        cas = list(prob["cascade"])
        self.h = gpmood_create(make_grid(prob), prob["gamma"], cas[0], prob["ell"],
                               make_options(prob, self.precision, eager))

    def close(self):
        if getattr(self, "h", None):
            gpmood_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        gpmood_set_stream(self.h, stream_ptr)

    def set_state(self, U):
        if not (hasattr(U, "data_ptr") and getattr(U, "is_cuda", False)):
            U = np.ascontiguousarray(U, dtype=np.float64)
            assert U.shape == (4, self.ny, self.nx), U.shape
        gpmood_set_state(self.h, U)

    def set_time(self, t):
        gpmood_set_time(self.h, t)

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((4, self.ny, self.nx))
        return gpmood_get_state(self.h, out)

    def step(self, cfl=None, want_dt=False):
        return gpmood_step(self.h, self.prob["cfl"] if cfl is None else cfl, want_dt)

    def step_dt(self, dt):
        gpmood_step_dt(self.h, dt)

    def run(self, t_end, cfl=None):
        return gpmood_run(self.h, t_end, self.prob["cfl"] if cfl is None else cfl)

    def step_async(self, cfl=None):
        """queue one step without waiting (errors surface at sync())"""
        gpmood_step_async(self.h, self.prob["cfl"] if cfl is None else cfl)

    def sync(self):
        gpmood_sync(self.h)

    def launch_count(self):
        return gpmood_launch_count(self.h)

    @property
    def nstages(self):
        return 5 if int(self.prob.get("rk", 3)) == 4 else 3

    def flags(self, maps=True):
        return gpmood_flags(self.h, self.nx, self.ny, maps, self.nstages)

    def last_launches(self):
        return gpmood_last_launches(self.h)

    def profile(self, enable=True):
        gpmood_profile(self.h, enable)

    # reverse mode: device pointers (ints) of caller-owned tensors
    def step_record(self, tape_ptr, otape_ptr, cfl=None, dt=0.0):
        out = C.c_double(0.0)
        cfl = (self.prob["cfl"] if cfl is None else cfl) if dt <= 0.0 else 0.0
        _check(load().gpmood_step_record(self.h, cfl, dt, C.c_void_p(tape_ptr),
                                         C.c_void_p(otape_ptr), C.byref(out)), "step_record")
        return out.value

    def state_tape_bytes(self):
        """device bytes of one recorded step's face-state tape"""
        n = C.c_size_t(0)
        _check(load().gpmood_state_tape_bytes(self.h, C.byref(n)), "state_tape_bytes")
        return n.value

    def step_record_states(self, tape_ptr, otape_ptr, stape_ptr, cfl=None, dt=0.0):
        out = C.c_double(0.0)
        cfl = (self.prob["cfl"] if cfl is None else cfl) if dt <= 0.0 else 0.0
        _check(load().gpmood_step_record_states(self.h, cfl, dt, C.c_void_p(tape_ptr),
                                                C.c_void_p(otape_ptr), C.c_void_p(stape_ptr),
                                                C.byref(out)), "step_record_states")
        return out.value

    def step_adjoint_states(self, tape_ptr, otape_ptr, stape_ptr, dt, t, lam_in_ptr,
                            lam_out_ptr):
        _check(load().gpmood_step_adjoint_states(self.h, C.c_void_p(tape_ptr),
                                                 C.c_void_p(otape_ptr), C.c_void_p(stape_ptr),
                                                 dt, t, C.c_void_p(lam_in_ptr),
                                                 C.c_void_p(lam_out_ptr)), "step_adjoint_states")

    def step_frozen(self, otape_ptr, dt):
        _check(load().gpmood_step_frozen(self.h, C.c_void_p(otape_ptr), dt), "step_frozen")

    def step_adjoint(self, tape_ptr, otape_ptr, dt, t, lam_in_ptr, lam_out_ptr):
        _check(load().gpmood_step_adjoint(self.h, C.c_void_p(tape_ptr), C.c_void_p(otape_ptr), dt,
                                          t, C.c_void_p(lam_in_ptr), C.c_void_p(lam_out_ptr)),
               "step_adjoint")

    def kernel_times(self):
        return gpmood_kernel_times(self.h)


class GPMoodBatch:
    """Many independent problems advanced together (gpmood_batch_* ABI).

    probs: problem dicts from ``inputs`` that share gamma, the cascade, the
    options and ell/dx, ell/dy."""

    def __init__(self, probs, precision="fp64", eager=False):
        self.probs = list(probs)
        self.n = len(self.probs)
        self.shapes = [(int(q["ny"]), int(q["nx"])) for q in self.probs]
        self.precision = FP32 if precision in ("fp32", FP32) else FP64
        grids = (Grid * self.n)(*[make_grid(q) for q in self.probs])
        ells = (C.c_double * self.n)(*[q["ell"] for q in self.probs])
        q0 = self.probs[0]
        opts = make_options(q0, self.precision, eager)
        h = C.c_void_p()
        _check(load().gpmood_batch_create(grids, self.n, q0["gamma"], list(q0["cascade"])[0],
                                          ells, C.byref(opts), C.byref(h)), "gpmood_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().gpmood_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        _check(load().gpmood_batch_set_stream(self.h, C.c_void_p(stream_ptr)), "set_stream")

    def _flat(self, Us):
        return np.ascontiguousarray(np.concatenate([np.asarray(U, dtype=np.float64).ravel()
                                                    for U in Us]))

    def set_state(self, Us):
        """Us: list of (4, ny, nx) arrays, or one flat concatenated array / CUDA tensor."""
        if hasattr(Us, "data_ptr") and getattr(Us, "is_cuda", False):
            _check(load().gpmood_batch_set_state(self.h, C.c_void_p(Us.data_ptr()), 1), "set_state")
            return
        flat = Us if isinstance(Us, np.ndarray) and Us.ndim == 1 else self._flat(Us)
        self._keep = flat
        _check(load().gpmood_batch_set_state(self.h, flat.ctypes.data_as(C.c_void_p), 0),
               "set_state")

    def get_state(self):
        total = sum(4 * ny * nx for ny, nx in self.shapes)
        flat = np.zeros(total)
        _check(load().gpmood_batch_get_state(self.h, flat.ctypes.data_as(C.c_void_p), 0),
               "get_state")
        out, off = [], 0
        for ny, nx in self.shapes:
            out.append(flat[off:off + 4 * ny * nx].reshape(4, ny, nx))
            off += 4 * ny * nx
        return out

    def step(self, cfl=None):
        _check(load().gpmood_batch_step(self.h, self.probs[0]["cfl"] if cfl is None else cfl),
               "gpmood_batch_step")

    def run(self, t_end, cfl=None):
        n = C.c_longlong(0)
        _check(load().gpmood_batch_run(self.h, t_end, self.probs[0]["cfl"] if cfl is None else cfl,
                                       C.byref(n)), "gpmood_batch_run")
        return n.value

    def info(self):
        t = np.zeros(self.n)
        dt = np.zeros(self.n)
        ns = np.zeros(self.n, dtype=np.int64)
        st = Stats()
        _check(load().gpmood_batch_info(self.h, t.ctypes.data_as(C.c_void_p),
                                        dt.ctypes.data_as(C.c_void_p),
                                        ns.ctypes.data_as(C.c_void_p), C.byref(st)), "info")
        return t, dt, ns, dict(iters=list(st.iters)[:3], nbad_first=list(st.nbad_first)[:3],
                               nbad_total=list(st.nbad_total)[:3])

    def tuning(self):
        w = (C.c_int * 2)()
        b = (C.c_int * 2)()
        rc = load().gpmood_batch_tuning(self.h, w, b)
        return (list(w), list(b)) if rc == 0 else None

    def grids(self):
        """(update-kernel blocks, MOOD-loop blocks) after the first step"""
        u, m = C.c_int(0), C.c_int(0)
        rc = load().gpmood_batch_grids(self.h, C.byref(u), C.byref(m))
        return (u.value, m.value) if rc == 0 else None

    def profile(self, enable=True):
        _check(load().gpmood_batch_profile(self.h, 1 if enable else 0), "profile")

    def kernel_times(self):
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
        _check(load().gpmood_batch_kernel_times(self.h, ms.ctypes.data_as(C.c_void_p),
                                                n.ctypes.data_as(C.c_void_p)), "kernel_times")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}
