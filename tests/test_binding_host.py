"""The binding's host arithmetic against the oracle, on the CPU: the witness loss and its gradient
with respect to the witness sums (what hq_sweep_adjoint is seeded with), and the emittance formed
from the eleven weighted moments that hq_beam_moments returns (same order as the oracle's)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import hq, inputs as I


@pytest.mark.parametrize("kind", ["mean", "mean+rms"])
@pytest.mark.parametrize("sums", [(-0.94, -0.10, -0.086), (-1.5, 0.3, -0.2), (2.0, 0.7, 0.9)])
def test_witness_loss_and_its_gradient_match_the_oracle(kind, sums):
    s = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in sums]
    res = O.SweepResult(witness={1: tuple(s)})
    L = O.witness_loss(res, 1, kind)
    L.backward()
    loss, grad = hq.witness_loss_grad(kind, *sums)
    assert loss == pytest.approx(float(L.detach()), rel=1e-14, abs=1e-15)
    for g, t in zip(grad, s):
        ref = 0.0 if t.grad is None else float(t.grad)   # "mean" does not depend on S2
        assert g == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_witness_loss_without_spread_keeps_a_finite_gradient():
    """All witness charge at one Ez: the spread term is zero and its derivative is dropped (the
    oracle's clamp at zero), not infinite."""
    s0, s1 = -2.0, -0.6
    loss, grad = hq.witness_loss_grad("mean+rms", s0, s1, s1 * s1 / s0)
    assert loss == pytest.approx(s1 / s0)
    assert all(np.isfinite(grad))


@pytest.mark.parametrize("seed", [0, 1])
def test_emittance_matches_the_oracle(seed):
    b = I.random_beam(20_000, 0.3, 0.4, 0.5, 1.0, energy_spread=1e-3, seed=1000 + seed)
    rng = np.random.default_rng(seed)
    b = dict(b, ux=rng.normal(0.0, 0.8, b["x"].size) + 0.3 * b["x"], uy=rng.normal(0.0, 0.5, b["x"].size))
    beam = O.as_beam(b)
    m = O.beam_moments(beam)
    ex, ey = hq.emittance(m)
    rx, ry = O.emittance(m)
    assert ex == pytest.approx(float(rx), rel=1e-12)
    assert ey == pytest.approx(float(ry), rel=1e-12)
    # and against numpy's weighted covariance of the particles themselves
    w = np.asarray(b["w"])
    cov = np.cov(np.stack([b["x"], b["ux"]]), aweights=w, bias=True)
    assert ex == pytest.approx(float(np.sqrt(np.linalg.det(cov))), rel=1e-9)
