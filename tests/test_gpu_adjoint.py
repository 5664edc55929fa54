"""Hand-written adjoint of the frozen-mask step (CUDA) against the oracle's
reference gradient (autograd of a plain PyTorch CPU restatement pinned to the
C oracle) and against central finite differences of the frozen-mask map."""
import numpy as np
import pytest

import oracle as O
import paper_2110_08683_gb300 as gp
from paper_2110_08683_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def recorded_step(g, U0, dt=0.0):
    ny, nx = g.ny, g.nx
    tape = torch.empty((3, 4, ny, nx), dtype=torch.float64, device="cuda")
    otape = torch.empty((3, ny, nx), dtype=torch.uint8, device="cuda")
    g.set_state(U0)
    dtv = g.step_record(tape.data_ptr(), otape.data_ptr(), dt=dt)
    torch.cuda.synchronize()
    return tape, otape, dtv


def vjp(g, tape, otape, dt, t, lam):
    lam = torch.as_tensor(lam, dtype=torch.float64, device="cuda").contiguous()
    out = torch.empty_like(lam)
    g.step_adjoint(tape.data_ptr(), otape.data_ptr(), dt, t, lam.data_ptr(), out.data_ptr())
    return out.cpu().numpy()


@pytest.mark.parametrize("case", ["shear", "quadrants", "wave"])
def test_single_step_vjp_matches_reference_gradient(case):
    from oracle.frozen_torch import FrozenStep

    if case == "shear":
        p = I.shear_layer(n=24, R=2, seed=3)
    elif case == "quadrants":
        p = I.quadrants(n=20, ny=17, R=3, seed=5)
    else:
        p = I.density_wave(nx=22, ny=19, amp=0.2, R=3, ell=0.1)
    g = gp.GPMood(p)
    tape, otape, dt = recorded_step(g, p["U0"])
    ords = otape.cpu().numpy()
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(p["U0"].shape)
    got = vjp(g, tape, otape, dt, 0.0, lam)
    fs = FrozenStep(p)
    U = torch.tensor(p["U0"], requires_grad=True)
    out = fs.step(U, ords, dt)
    (ref,) = torch.autograd.grad((out * torch.tensor(lam)).sum(), U)
    ref = ref.numpy()
    assert np.isfinite(ref).all()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_rollout_gradient_against_frozen_finite_differences():
    from paper_2110_08683_gb300.autograd import rollout

    p = I.shear_layer(n=32, R=2, seed=0)
    g = gp.GPMood(p)
    n = 32
    U0 = torch.tensor(p["U0"], device="cuda")
    region = np.zeros((n, n))
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c, indexing="xy")
    region[(X >= 0.4) & (X <= 0.6) & (Y >= 0.4) & (Y <= 0.6)] = 1.0 / n**2
    W = torch.zeros((4, n, n), dtype=torch.float64, device="cuda")
    W[0] = torch.tensor(region)
    nsteps, every = 10, 4
    U0r = U0.clone().requires_grad_()
    UN = rollout(U0r, g, nsteps, every=every)
    J = (UN * W).sum()
    J.backward()
    grad = U0r.grad.cpu().numpy()
    # the frozen-mask map: record the forward's radii and dt's, replay them
    tapes = []
    g.set_state(p["U0"])
    for _ in range(nsteps):
        tape = torch.empty((3, 4, n, n), dtype=torch.float64, device="cuda")
        otape = torch.empty((3, n, n), dtype=torch.uint8, device="cuda")
        dt = g.step_record(tape.data_ptr(), otape.data_ptr())
        tapes.append((otape, dt))

    def J_frozen(U):
        g.set_state(U)
        for otape, dt in tapes:
            g.step_frozen(otape.data_ptr(), dt)
        return float((torch.tensor(g.get_state(), device="cuda") * W).sum())

    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(6):
        d = rng.standard_normal(p["U0"].shape)
        fd = (J_frozen(p["U0"] + h * d) - J_frozen(p["U0"] - h * d)) / (2 * h)
        ad = float((grad * d).sum())
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-12), (ad, fd)


def test_fp32_adjoint_close_to_fp64():
    p = I.shear_layer(n=32, R=2, seed=0)
    rng = np.random.default_rng(2)
    lam = rng.standard_normal(p["U0"].shape)
    res = {}
    for prec in ("fp64", "fp32"):
        g = gp.GPMood(p, prec)
        tape, otape, dt = recorded_step(g, p["U0"], dt=1e-3)
        res[prec] = vjp(g, tape, otape, 1e-3, 0.0, lam)
    rel = np.abs(res["fp32"] - res["fp64"]).max() / np.abs(res["fp64"]).max()
    assert rel <= 1e-4, rel


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resident_tapes_and_recomputed_segments_agree(precision):
    """The forward that records every step's tape runs the same kernels as
    the plain step, and the reverse pass over resident tapes equals the one
    that steps the segments again from checkpoints, bit for bit, whether the
    re-recorded segments keep their face states (the adjoint then reads
    them) or not (the adjoint reconstructs them): quadrant problem, MOOD
    lowers radii, so the frozen masks are not uniform and the MOOD loop's
    recomputed faces reach the state tape too."""
    from paper_2110_08683_gb300.autograd import rollout

    p = I.quadrants(n=40, ny=36, R=3, seed=2)
    g = gp.GPMood(p, precision)
    U0 = torch.tensor(p["U0"], device="cuda")
    nsteps = 7
    g.set_state(p["U0"])
    for _ in range(nsteps):
        g.step()
    plain = torch.tensor(g.get_state(), device="cuda")
    rng = np.random.default_rng(4)
    W = torch.tensor(rng.standard_normal(p["U0"].shape), device="cuda")
    outs, grads = [], []
    for every, budget, states in ((None, None, True), (3, None, True), (3, None, False),
                                  (None, 1, True)):
        U0r = U0.clone().requires_grad_()
        UN = rollout(U0r, g, nsteps, every=every, budget=budget, states=states)
        (UN * W).sum().backward()
        outs.append(UN.detach().clone())
        grads.append(U0r.grad.clone())
    assert torch.equal(outs[0], plain)
    for k in (1, 2, 3):
        assert torch.equal(outs[k], outs[0])
        assert torch.equal(grads[k], grads[0])
    assert torch.isfinite(grads[0]).all()
