"""The oracle's taped FP64 adjoint (reverse-mode autograd through the sweep) against
central finite differences (step 1e-6, relative to the parameter scale).

This pins the gradient reference the GPU adjoint is compared with: beam weights
(random directions), the plasma density scale n0 and a radial density profile entry,
for both witness losses (mean Ez and mean + RMS spread)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2109_10277_gb300 import inputs as I


def setup(nz=24, order=1):
    g = dict(nx=24, ny=24, nzeta=nz, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0, zeta_min=-7.0, zeta_max=5.0,
             shape_order=order, n_pc_iter=2, pc_mix=0.05, psi_guard=0.02,
             radial_profile=[1.0, 1.0, 0.8, 0.5, 0.3], profile_rmax=8.5)
    d = I.fixed_ppc_beam(g, 0.8, 1.0, 2.0)
    w = I.fixed_ppc_beam(g, 0.5, 0.6, 10.0, zeta0=-3.0, gamma=I.GAMMA_WITNESS)
    return g, d, w


def loss_fn(g, d, w, kind):
    sp = O.GridSpec(**g)

    def f(wd, ww, n0, prof):
        bd, bw = O.as_beam(d), O.as_beam(w)
        bd["w"], bw["w"] = wd, ww
        r = O.sweep(sp, [bd, bw], witness=(1,), record=(), n0_scale=n0, radial_profile=prof)
        return O.witness_loss(r, 1, kind)
    return f


@pytest.mark.parametrize("kind,order", [("mean", 1), ("mean+rms", 2)])
def test_taped_adjoint_matches_central_fd(kind, order):
    g, d, w = setup(order=order)
    f = loss_fn(g, d, w, kind)
    wd = torch.tensor(d["w"], dtype=torch.float64, requires_grad=True)
    ww = torch.tensor(w["w"], dtype=torch.float64, requires_grad=True)
    n0 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor(g["radial_profile"], dtype=torch.float64, requires_grad=True)
    L = f(wd, ww, n0, prof)
    L.backward()
    rng = np.random.default_rng(5)
    h = 1e-6
    base = [wd.detach(), ww.detach(), n0.detach(), prof.detach()]

    def fd(k, v):
        args_p = [b + (h * v if i == k else 0) for i, b in enumerate(base)]
        args_m = [b - (h * v if i == k else 0) for i, b in enumerate(base)]
        with torch.no_grad():
            return float((f(*args_p) - f(*args_m)) / (2 * h))

    for k, grad in ((0, wd.grad), (1, ww.grad)):
        v = torch.tensor(rng.standard_normal(base[k].shape[0]), dtype=torch.float64) * base[k]
        a, b = float((grad * v).sum()), fd(k, v)
        assert abs(a - b) <= 1e-6 * abs(b), (k, a, b)
    a, b = float(n0.grad), fd(2, torch.tensor(1.0, dtype=torch.float64))
    assert abs(a - b) <= 1e-6 * abs(b), ("n0", a, b)
    e = torch.zeros_like(base[3])
    e[2] = 1.0
    a, b = float(prof.grad[2]), fd(3, e)
    assert abs(a - b) <= 1e-6 * abs(b) + 1e-12, ("profile[2]", a, b)
