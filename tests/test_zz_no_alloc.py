"""The allocation-free step (gpmood_step_noalloc) against the ordinary handle
path, on two calls in a row, in FP64 and in FP32.

gpmood_step_noalloc serves callers that cannot allocate device memory while
they run (a framework that owns the device memory pool, a real-time loop that
must not allocate after start-up): its buffers live in one static device
array of the library.  Both paths launch the same kernels on the same data,
so their results must agree bit for bit.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def two_steps_both_ways(p, precision):
    torch = pytest.importorskip("torch")
    # the ordinary path: a handle with its own device buffers
    h = gp.GPMood(p, precision)
    h.set_state(p["U0"])
    dt1 = h.step(want_dt=True)
    ref1 = h.get_state()
    dt2 = h.step(want_dt=True)
    ref2 = h.get_state()
    h.close()
    # the allocation-free path; the caller owns input and output
    prec = gp.FP32 if precision == "fp32" else gp.FP64
    u_in = torch.tensor(p["U0"], dtype=torch.float64, device="cuda")
    u_mid = torch.empty_like(u_in)
    u_out = torch.empty_like(u_in)
    torch.cuda.synchronize()
    da = gp.gpmood_step_noalloc(p, u_in.data_ptr(), u_mid.data_ptr(), 0.0, p["cfl"],
                                precision=prec)
    db = gp.gpmood_step_noalloc(p, u_mid.data_ptr(), u_out.data_ptr(), da, p["cfl"],
                                precision=prec)
    torch.cuda.synchronize()
    assert da == dt1 and db == dt2
    np.testing.assert_array_equal(u_mid.cpu().numpy(), ref1)
    np.testing.assert_array_equal(u_out.cpu().numpy(), ref2)
    # the input was not modified
    np.testing.assert_array_equal(u_in.cpu().numpy(), p["U0"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_step_matches_handle_step_twice(precision):
    # shocks: the MOOD loop runs in every stage
    two_steps_both_ways(I.quadrants(n=48, ny=40, R=3, seed=7), precision)


def test_noalloc_fp32_grid_near_the_scratch_limit():
    """256 x 256 at R = 3 in FP32, the largest square grid that fits, fills
    99.7% of the scratch (three states, their float shadows, fluxes, maps,
    stamps and queues)."""
    two_steps_both_ways(I.quadrants(n=256, R=3, seed=3), "fp32")


def test_noalloc_rejects_grids_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    u = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    for p, prec in ((I.vortex(n=512, R=3), gp.FP64), (I.quadrants(n=264, R=3, seed=1), gp.FP32)):
        with pytest.raises(gp.GpmoodError) as e:
            gp.gpmood_step_noalloc(p, u.data_ptr(), u.data_ptr(), 0.0, 0.8, precision=prec)
        assert e.value.code == -8
