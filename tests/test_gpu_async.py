"""Queued (asynchronous) steps through the C ABI: gpmood_step_async queues a
step graph that opens with a gate and returns without reading anything back;
gpmood_sync settles the buffer rotation from the device's step count.
Queued steps must equal waited-for steps bit for bit, run() (which queues in
chunks and lets the gate stop at t_end) must equal the eager run, and a
failure must stop the steps queued after it."""
import numpy as np
import pytest

import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _quads(rk=3):
    p = I.quadrants(n=48, ny=40, R=3, seed=1)
    p["rk"] = rk
    return p


@pytest.mark.parametrize("rk", [3, 4])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_queued_steps_equal_waited_steps(precision, rk):
    p = _quads(rk)
    a, b = gp.GPMood(p, precision), gp.GPMood(p, precision)
    a.set_state(p["U0"])
    b.set_state(p["U0"])
    for _ in range(6):
        a.step()
        b.step_async()
    b.sync()
    oa, fa, sa = a.flags()
    ob, fb, sb = b.flags()
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(oa, ob) and np.array_equal(fa, fb)
    assert sa["t"] == sb["t"] and sa["nsteps"] == sb["nsteps"] == 6
    assert sa["iters"] == sb["iters"] and sum(sa["nbad_first"]) > 0
    # a waited-for step after queued ones continues from the settled rotation
    a.step()
    b.step()
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chunked_run_equals_eager_run(precision):
    """run() on a graph handle queues chunks of steps past t_end (the gate
    makes the surplus no-ops); the eager handle steps one at a time."""
    p = I.quadrants(n=40, R=2, seed=4)
    res = []
    for eager in (False, True):
        g = gp.GPMood(p, precision, eager=eager)
        g.set_state(p["U0"])
        n1 = g.run(0.05)
        n2 = g.run(0.11)
        st = g.flags(maps=False)[2]
        res.append((g.get_state(), n1, n2, st["t"], st["nsteps"]))
        g.close()
    (Ug, g1, g2, tg, ng), (Ue, e1, e2, te, ne) = res
    assert (g1, g2, ng) == (e1, e2, ne) and g1 > 3 and g2 > 3
    assert tg == te == 0.11
    assert np.array_equal(Ug, Ue)


def test_failure_stops_the_queued_steps():
    """The MOOD cap at the first step: the steps queued after it do nothing,
    sync reports the cap, and the state, time and step count are those
    before the failed step (as after a waited-for failed step)."""
    p = I.quadrants(n=32, R=3, seed=1)
    p["max_iters"] = 1
    g = gp.GPMood(p)
    g.set_state(p["U0"])
    for _ in range(3):
        g.step_async()
    with pytest.raises(gp.GpmoodError) as e:
        g.sync()
    assert e.value.code == -5
    st = g.flags(maps=False)[2]
    assert st["t"] == 0.0 and st["nsteps"] == 0
    assert np.array_equal(g.get_state(), p["U0"])
    # the handle recovers with a new state
    p2 = I.quadrants(n=32, R=3, seed=1)
    g2 = gp.GPMood(p2)
    g2.set_state(p2["U0"])
    g2.step()
    g.set_state(p2["U0"])
    with pytest.raises(gp.GpmoodError):
        g.step()  # the cap is still one iteration
    g.close()
    g2.close()


@pytest.mark.parametrize("problem", ["vortex", "quadrants"])
def test_launch_count_is_counted_on_the_device(problem):
    # every step launches the gate, the two time-step kernels, the ghost fill
    # of the first stage's input, three kernels a stage (the x and y faces in
    # one kernel, update, the MOOD loop, which fills the next stage's ghosts
    # or reduces the next step's CFL rate) and the finishing one, whether
    # MOOD iterates (quadrants) or not (the vortex)
    p = I.vortex(n=64, R=3) if problem == "vortex" else I.quadrants(n=64, R=3, seed=4)
    g = gp.GPMood(p)
    g.set_state(p["U0"])
    n0 = g.launch_count()
    for _ in range(5):
        g.step_async()
    g.sync()
    assert g.launch_count() - n0 == 5 * (1 + 2 + 1 + 3 * 3 + 1)
    if problem == "quadrants":
        assert sum(g.flags(maps=False)[2]["iters"]) > 0
    g.close()


@pytest.mark.parametrize("eager", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_programmatic_launch_equals_stream_order(precision, eager):
    """Programmatic dependent launch only overlaps the scheduling of a
    kernel with the end of its predecessor (every step kernel waits for its
    predecessor before touching memory): bit-identical results to plain
    stream order, MOOD iterations included."""
    p = _quads()
    out = []
    for serial in (0, 1):
        q = dict(p, serial_launch=serial)
        g = gp.GPMood(q, precision, eager=eager)
        g.set_state(q["U0"])
        for _ in range(4):
            g.step_async()
        g.sync()
        o, f, st = g.flags()
        out.append((g.get_state(), o, f, st))
        g.close()
    (U0, o0, f0, s0), (U1, o1, f1, s1) = out
    assert np.array_equal(U0, U1) and np.array_equal(o0, o1) and np.array_equal(f0, f1)
    assert s0["iters"] == s1["iters"] and sum(s0["nbad_first"]) > 0


@pytest.mark.parametrize("R", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_face_kernel_equals_the_two_sweeps(precision, R):
    """The first-pass face kernel that solves x and y faces in one launch
    (each cell forming its stencil sums once) gives the same fluxes, bit for
    bit, as one kernel per direction: equal states, radii and MOOD counters
    after several steps with MOOD active, on a grid with ragged segments
    and bands in both directions."""
    p = I.quadrants(n=71, ny=45, R=R, seed=9)
    out = []
    for split in (0, 1):
        q = dict(p, split_faces=split)
        g = gp.GPMood(q, precision)
        g.set_state(q["U0"])
        for _ in range(3):
            g.step()
        o, f, st = g.flags()
        out.append((g.get_state(), o, f, st))
        g.close()
    (U0, o0, f0, s0), (U1, o1, f1, s1) = out
    assert np.array_equal(U0, U1) and np.array_equal(o0, o1) and np.array_equal(f0, f1)
    assert s0["iters"] == s1["iters"] and sum(s0["nbad_first"]) > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_state_io_through_pinned_host_memory(precision):
    """set_state / get_state on page-locked host buffers go through one
    kernel that reads or writes the host memory directly; pageable buffers
    through the CUDA driver's staged copies.  Both give the same steps."""
    torch = pytest.importorskip("torch")
    p = _quads()
    shape = p["U0"].shape
    Up = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    Up[...] = p["U0"]
    a, b = gp.GPMood(p, precision), gp.GPMood(p, precision)
    a.set_state(p["U0"])
    b.set_state(Up)
    for _ in range(2):
        a.step()
        b.step()
    Oa = a.get_state()
    Ob = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    b.get_state(Ob)
    assert np.array_equal(Oa, Ob)
    # and back in from the pinned result
    b.set_state(Ob)
    assert np.array_equal(b.get_state(), Oa)
    a.close()
    b.close()
