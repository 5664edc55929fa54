"""The C ABI library builds, loads and exports every entry point that
include/gpmood.h declares (no GPU needed: nothing is called but strerror)."""
import ctypes
import os
import re

import pytest

import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*|void)\s+(gpmood_\w+)\s*\(", txt, re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert {"gpmood_create", "gpmood_set_state", "gpmood_step", "gpmood_run", "gpmood_flags",
            "gpmood_destroy"} <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def test_strerror_without_a_device():
    lib = gp.load()
    assert lib.gpmood_strerror(-5) == b"MOOD iteration cap reached"
    assert lib.gpmood_strerror(0) == b"ok"


def test_create_rejects_bad_arguments_before_touching_the_device():
    from paper_2110_08683_gb300 import inputs as I

    p = I.vortex(n=16, R=3)
    p["nx"] = 2  # fewer cells than ghost layers
    g = gp.make_grid(p)
    o = gp.make_options(p)
    h = ctypes.c_void_p()
    rc = gp.load().gpmood_create(ctypes.byref(g), 1.4, 3, 0.5, ctypes.byref(o), ctypes.byref(h))
    assert rc == -1 and not h.value
    p = I.vortex(n=16, R=3)
    p["cascade"] = [3, 3, 0]
    o = gp.make_options(p)
    rc = gp.load().gpmood_create(ctypes.byref(gp.make_grid(p)), 1.4, 3, 0.5, ctypes.byref(o),
                                 ctypes.byref(h))
    assert rc == -1


def test_batch_binding_marshals_and_rejects_mixed_weights():
    # problems that would need different GP weights (ell/dx differs): the
    # library refuses before touching the device
    from paper_2110_08683_gb300 import inputs as I

    a = I.quadrants(n=16, R=2, seed=1)
    b = I.quadrants(n=24, R=2, seed=2)
    b["ell"] = 2.0 * b["ell"]
    with pytest.raises(gp.GpmoodError) as e:
        gp.GPMoodBatch([a, b])
    assert e.value.code == -1


def test_create_rejects_poly3_beyond_radius_one_before_touching_the_device():
    # POL-MOOD3 is the cascade Poly3 -> FOG: R_max must be 1; unknown
    # reconstruction codes are refused too
    from paper_2110_08683_gb300 import inputs as I

    p = I.vortex(n=16, R=3)
    p["recon"] = "poly3"
    h = ctypes.c_void_p()
    rc = gp.load().gpmood_create(ctypes.byref(gp.make_grid(p)), 1.4, 3, 0.5,
                                 ctypes.byref(gp.make_options(p)), ctypes.byref(h))
    assert rc == -1 and not h.value
    o = gp.make_options(I.vortex(n=16, R=1, cascade=[1, 0]))
    o.recon = 7
    rc = gp.load().gpmood_create(ctypes.byref(gp.make_grid(p)), 1.4, 1, 0.5, ctypes.byref(o),
                                 ctypes.byref(h))
    assert rc == -1 and not h.value


def test_noalloc_rejects_what_create_rejects_before_touching_the_device():
    # only SSP-RK3 (rk 0 or 3) and two-dimensional grids (dim 0 or 2); the
    # checks run before any CUDA call, so no device is needed
    from paper_2110_08683_gb300 import inputs as I

    p = I.quadrants(n=16, R=2, seed=1)
    lib = gp.load()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the call fails first
    dt = ctypes.c_double(0.0)

    def call(g, o):
        return lib.gpmood_step_noalloc(ctypes.byref(g), 1.4, 2, p["ell"], ctypes.byref(o), dummy,
                                       dummy, 0.0, 0.8, ctypes.byref(dt), None)

    for rk in (1, 2, 4, 5):
        o = gp.make_options(p)
        o.rk = rk
        assert call(gp.make_grid(p), o) == -1, rk
    for dim in (1, 3, 7, -1):
        g = gp.make_grid(p)
        g.dim = dim
        assert call(g, gp.make_options(p)) == -1, dim
