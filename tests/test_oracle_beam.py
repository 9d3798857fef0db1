"""Pins for the oracle's beam deposit (Sec. 3.1 per-slice beam deposition; order 0
longitudinally, orders 0-3 transversely).

The expected values are closed forms of the physics, not the oracle's own formula:
  * a beam of macroparticles placed one per (cell, slice) at the centres, each carrying
    the number of physical particles n_b(x, y, zeta) dx dy dzeta of its cell, must
    deposit the charge density q n_b at every interior node.  For an affine density
    this holds exactly (a cardinal B-spline sampled symmetrically about a node sums to
    one and has zero first moment), so the 1/(dx dy dzeta) normalisation is fixed;
  * a beam in which every particle has the same momentum u carries the current
    J = rho v with v = u / sqrt(1 + |u|^2) (the relativistic velocity, c = 1);
  * the charge a random beam deposits on a slice, summed over the nodes and multiplied
    by the cell volume, is q times the weight of the particles binned into it.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O


def grid(order):
    return O.GridSpec(nx=20, ny=16, nzeta=6, xmin=-2.5, xmax=2.5, ymin=-1.6, ymax=2.4,
                      zeta_min=-1.0, zeta_max=2.0, shape_order=order)


def lattice_beam(sp, density, u=(0.0, 0.0, 50.0), charge=-1.0):
    """One macroparticle per (cell, slice) at its centre with weight density(x, y, zeta) dx dy dzeta."""
    xc = sp.xmin + (np.arange(sp.nx) + 0.5) * sp.dx
    yc = sp.ymin + (np.arange(sp.ny) + 0.5) * sp.dy
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    x, y, z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    n = x.size
    w = density(x, y, z) * sp.dx * sp.dy * sp.dzeta
    return O.as_beam(dict(x=x, y=y, zeta=z, ux=np.full(n, u[0]), uy=np.full(n, u[1]), uz=np.full(n, u[2]), w=w,
                          charge=charge))


def slice_members(sp, beam, i):
    off, order = O.beam_csr(sp, O.beam_bins(sp, beam["zeta"]))
    return order[off[i]:off[i + 1]]


@pytest.mark.parametrize("order", [1, 2, 3])
def test_beam_density_is_q_n_b_at_nodes(order):
    sp = grid(order)
    a, bx, by, bz = 3.0, 0.4, -0.7, 0.25
    dens = lambda x, y, z: a + bx * x + by * y + bz * z  # noqa: E731  affine, positive on the box
    beam = lattice_beam(sp, dens)
    zc = sp.zeta_max - (np.arange(sp.nzeta) + 0.5) * sp.dzeta
    m = order + 1  # nodes whose whole stencil support lies on populated cells
    xs = sp.xmin + np.arange(sp.nx) * sp.dx
    ys = sp.ymin + np.arange(sp.ny) * sp.dy
    for i in range(sp.nzeta):
        (rho,) = O.beam_deposit_slice(sp, beam, slice_members(sp, beam, i), ("rho",))
        expect = -dens(xs[None, :], ys[:, None], zc[i])
        got = rho.numpy()
        assert np.allclose(got[m:sp.ny - m, m:sp.nx - m], expect[m:sp.ny - m, m:sp.nx - m], rtol=0, atol=1e-12), i


def test_beam_density_ngp_constant():
    """Order 0 samples a single cell centre per node: exact for a uniform density."""
    sp = grid(0)
    beam = lattice_beam(sp, lambda x, y, z: np.full_like(x, 2.5))
    (rho,) = O.beam_deposit_slice(sp, beam, slice_members(sp, beam, 2), ("rho",))
    assert np.allclose(rho.numpy()[1:, 1:], -2.5, rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", [1, 3])
def test_beam_current_is_rho_times_velocity(order):
    sp = grid(order)
    u = (3.0, -2.0, 40.0)
    beam = lattice_beam(sp, lambda x, y, z: 1.5 + 0.2 * x, u=u)
    gam = math.sqrt(1.0 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    v = [c / gam for c in u]
    rho, jx, jy, jz = O.beam_deposit_slice(sp, beam, slice_members(sp, beam, 3))
    for j, vc in zip((jx, jy, jz), v):
        assert torch.allclose(j, rho * vc, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("order", [0, 2])
def test_random_beam_slice_charge(order):
    sp = grid(order)
    rng = np.random.Generator(np.random.PCG64(77))
    n = 4000
    x = 0.35 * rng.standard_normal(n)
    y = 0.2 + 0.35 * rng.standard_normal(n)
    z = 0.5 + 0.6 * rng.standard_normal(n)
    w = rng.uniform(0.5, 1.5, n)
    beam = O.as_beam(dict(x=x, y=y, zeta=z, ux=np.zeros(n), uy=np.zeros(n), uz=np.full(n, 100.0), w=w, charge=-2.0))
    vol = sp.dx * sp.dy * sp.dzeta
    for i in range(sp.nzeta):
        t = np.floor((sp.zeta_max - z) / sp.dzeta)
        inside = (t == i) & (np.abs(x) < 2.5 - 3 * sp.dx) & (y > -1.6 + 3 * sp.dy) & (y < 2.4 - 3 * sp.dy)
        sel = torch.as_tensor(np.nonzero(inside)[0])
        (rho,) = O.beam_deposit_slice(sp, beam, sel, ("rho",))
        q = -2.0 * float(w[inside].sum())
        assert abs(float(rho.sum()) * vol - q) <= 1e-12 * max(1.0, abs(q)), i


def test_beam_emittance_against_weighted_covariance():
    """The oracle's emittance from raw moments equals sqrt(det) of numpy's weighted covariance
    of (x, ux) and (y, uy); it is invariant under a linear shear u -> u + a x (a thin lens) and
    under a centroid offset, and scales with the spread of the uncorrelated part."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 5000
    x = 0.3 * rng.standard_normal(n) + 0.5
    y = 0.2 * rng.standard_normal(n) - 0.1
    ux = 0.01 * rng.standard_normal(n) + 0.2 * x
    uy = 0.02 * rng.standard_normal(n)
    w = rng.uniform(0.2, 1.0, n)
    b = O.as_beam(dict(x=x, y=y, zeta=np.zeros(n), ux=ux, uy=uy, uz=np.full(n, 1e3), w=w))
    ex, ey = O.emittance(O.beam_moments(b))
    for e, (a, c) in ((ex, (x, ux)), (ey, (y, uy))):
        cov = np.cov(np.vstack([a, c]), aweights=w, bias=True)
        assert abs(e - math.sqrt(np.linalg.det(cov))) <= 1e-10 * e
    b2 = dict(b)
    b2["ux"] = b["ux"] + 3.0 * b["x"]
    b2["x"] = b["x"] + 7.0
    ex2, _ = O.emittance(O.beam_moments(b2))
    assert abs(ex2 - ex) <= 1e-8 * ex
    b3 = dict(b)
    b3["ux"] = 0.2 * b["x"] + 2.0 * (b["ux"] - 0.2 * b["x"])
    ex3, _ = O.emittance(O.beam_moments(b3))
    assert abs(ex3 - 2.0 * ex) <= 1e-8 * ex
