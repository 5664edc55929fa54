"""The allocation-free step (gpmood_step_noalloc) against the ordinary handle
path, on two calls in a row.

gpmood_step_noalloc serves callers that cannot allocate device memory while
they run (a framework that owns the device memory pool, a real-time loop that
must not allocate after start-up): its buffers live in one static device
array of the library.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(4))


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    p = I.quadrants(n=48, ny=40, R=3, seed=7)
    # the ordinary path: a handle with its own device buffers
    h = gp.GPMood(p)
    h.set_state(p["U0"])
    dt1 = h.step(want_dt=True)
    ref1 = h.get_state()
    dt2 = h.step(want_dt=True)
    ref2 = h.get_state()
    h.close()
    # the allocation-free path; the caller owns input and output
    u_in = torch.tensor(p["U0"], dtype=torch.float64, device="cuda")
    u_mid = torch.empty_like(u_in)
    u_out = torch.empty_like(u_in)
    torch.cuda.synchronize()
    da = gp.gpmood_step_noalloc(p, u_in.data_ptr(), u_mid.data_ptr(), 0.0, p["cfl"])
    db = gp.gpmood_step_noalloc(p, u_mid.data_ptr(), u_out.data_ptr(), da, p["cfl"])
    torch.cuda.synchronize()
    assert abs(da - dt1) <= 1e-14 * dt1 and abs(db - dt2) <= 1e-14 * dt2
    assert relerr(u_mid.cpu().numpy(), ref1) <= 1e-12
    assert relerr(u_out.cpu().numpy(), ref2) <= 1e-12
    # the input was not modified
    np.testing.assert_array_equal(u_in.cpu().numpy(), p["U0"])


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    p = I.vortex(n=512, R=3)
    u = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(gp.GpmoodError) as e:
        gp.gpmood_step_noalloc(p, u.data_ptr(), u.data_ptr(), 0.0, 0.8)
    assert e.value.code == -8
