"""Pins of the oracle-side reference for gradients: the plain PyTorch CPU
restatement of the frozen-radius step reproduces the C oracle's step, and its
autograd gradient agrees with central finite differences."""
import numpy as np
import pytest

import oracle as O
from paper_2110_08683_gb300 import inputs as I

torch = pytest.importorskip("torch")
from oracle.frozen_torch import FrozenStep  # noqa: E402


@pytest.mark.parametrize("case", ["quadrants", "shear", "wave_outflow"])
def test_forward_matches_c_oracle(case):
    if case == "quadrants":
        p = I.quadrants(n=20, ny=17, R=3, seed=5)
    elif case == "shear":
        p = I.shear_layer(n=24, R=2, seed=1)
    else:
        p = I.density_wave(nx=18, ny=16, amp=0.2, R=2, ell=0.1)
        p["bc"] = ["outflow", "outflow", "reflect", "reflect"]
    o = O.Oracle(p)
    U1, st, ords, _ = o.step(p["U0"], 0.0)
    out = FrozenStep(p).step(torch.tensor(p["U0"]), ords, st["dt"]).numpy()
    assert np.abs(out - U1).max() <= 1e-14 * np.abs(U1).max()
    if case == "quadrants":
        assert sum(st["nbad_first"]) > 0  # radii below the top in play


@pytest.mark.parametrize("case", ["quadrants", "shear"])
def test_gradient_matches_central_differences(case):
    p = I.quadrants(n=14, ny=12, R=3, seed=5) if case == "quadrants" else I.shear_layer(n=16, R=2)
    o = O.Oracle(p)
    _, st, ords, _ = o.step(p["U0"], 0.0)
    fs = FrozenStep(p)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(p["U0"].shape)
    U = torch.tensor(p["U0"], requires_grad=True)
    J = (fs.step(U, ords, st["dt"]) * torch.tensor(lam)).sum()
    (grad,) = torch.autograd.grad(J, U)
    # the frozen-radius map is piecewise smooth: HLLC's min/max wave speeds and
    # contact-side choice have kinks, which a finite difference straddles
    # with a probability that grows with h; discontinuous data need a small h
    h, tol = (1e-8, 1e-6) if case == "quadrants" else (1e-6, 1e-7)
    for _ in range(4):
        d = rng.standard_normal(p["U0"].shape)
        Jp = float((fs.step(torch.tensor(p["U0"] + h * d), ords, st["dt"]) * torch.tensor(lam)).sum())
        Jm = float((fs.step(torch.tensor(p["U0"] - h * d), ords, st["dt"]) * torch.tensor(lam)).sum())
        fd = (Jp - Jm) / (2 * h)
        assert abs(float((grad * torch.tensor(d)).sum()) - fd) <= tol * abs(fd)
