"""Pins for the oracle's fast Poisson solver and finite differences (Sec. 3.2, DST-I).

Each check compares against something other than the oracle's own formula:
explicit sine sums, the 5-point stencil written out with loops, the orthogonality
of DST-I, and polynomials whose central differences are exact.
"""
import math

import pytest
import torch

import oracle as O


def spec(nx=12, ny=10, Lx=3.0, Ly=2.0):
    # dx != dy and nx != ny so that a transposed operand or swapped axis fails
    return O.GridSpec(nx=nx, ny=ny, nzeta=4, xmin=-Lx / 2, xmax=Lx / 2 + 0.7, ymin=-Ly / 2,
                      ymax=Ly / 2, zeta_min=0.0, zeta_max=1.0)


def stencil_loops(sp, f):
    """5-point Laplacian on interior nodes, wall nodes (0 and n) read as zero."""
    out = torch.zeros(sp.ny, sp.nx, dtype=torch.float64)

    def val(i, j):
        if i <= 0 or j <= 0 or i >= sp.ny or j >= sp.nx:
            return 0.0
        return float(f[i, j])

    for i in range(1, sp.ny):
        for j in range(1, sp.nx):
            out[i, j] = ((val(i, j + 1) - 2 * val(i, j) + val(i, j - 1)) / sp.dx ** 2
                         + (val(i + 1, j) - 2 * val(i, j) + val(i - 1, j)) / sp.dy ** 2)
    return out


@pytest.mark.parametrize("n", [8, 12, 17])
def test_dst_orthogonality(n):
    S = O.dst_matrix(n)
    P = S @ S
    eye = torch.eye(n, dtype=torch.float64) * (n / 2.0)
    eye[0, 0] = 0.0
    assert torch.allclose(P, eye, atol=1e-12 * n)


def test_dst2_brute_force():
    sp = spec(nx=7, ny=6)
    g = torch.Generator().manual_seed(3)
    a = torch.randn(sp.ny, sp.nx, generator=g, dtype=torch.float64)
    got = O.dst2(sp, a)
    ref = torch.zeros_like(a)
    for l in range(sp.ny):
        for k in range(sp.nx):
            s = 0.0
            for i in range(1, sp.ny):
                for j in range(1, sp.nx):
                    s += float(a[i, j]) * math.sin(math.pi * i * l / sp.ny) * math.sin(math.pi * j * k / sp.nx)
            ref[l, k] = s
    assert torch.allclose(got, ref, atol=1e-12)


def test_poisson_eigenmode():
    sp = spec()
    jx = torch.arange(sp.nx, dtype=torch.float64)
    iy = torch.arange(sp.ny, dtype=torch.float64)
    for k, l in ((1, 1), (3, 2), (sp.nx - 1, sp.ny - 1), (5, 1)):
        mode = torch.sin(math.pi * l * iy / sp.ny)[:, None] * torch.sin(math.pi * k * jx / sp.nx)[None, :]
        lap = stencil_loops(sp, mode)
        # the mode is an eigenvector of the written-out stencil ...
        ratio = lap[1:, 1:] / mode[1:, 1:]
        lam = float(ratio.median())
        mask = mode[1:, 1:].abs() > 1e-6
        assert torch.allclose(ratio[mask], torch.full_like(ratio[mask], lam), rtol=1e-10)
        # ... and the solver inverts it exactly
        f = O.poisson_solve(sp, mode)
        assert torch.allclose(f, mode / lam, atol=1e-12 * mode.abs().max() / abs(lam))


def test_poisson_residual_random():
    sp = spec(nx=16, ny=11)
    g = torch.Generator().manual_seed(7)
    s = torch.randn(sp.ny, sp.nx, generator=g, dtype=torch.float64)
    s[0, :] = 0.0
    s[:, 0] = 0.0
    f = O.poisson_solve(sp, s)
    assert torch.all(f[0, :] == 0) and torch.all(f[:, 0] == 0)
    r = stencil_loops(sp, f)
    assert float((r - s).abs().max()) <= 1e-11 * float(s.abs().max())


def test_central_differences_exact_on_quadratics():
    sp = spec()
    x = sp.xmin + torch.arange(sp.nx, dtype=torch.float64) * sp.dx
    y = sp.ymin + torch.arange(sp.ny, dtype=torch.float64) * sp.dy
    # quadratics vanishing on both walls: central differences are exact everywhere inside
    fx = ((x - sp.xmin) * (sp.xmax - x))[None, :].expand(sp.ny, sp.nx).clone()
    fy = ((y - sp.ymin) * (sp.ymax - y))[:, None].expand(sp.ny, sp.nx).clone()
    dfx = (sp.xmax + sp.xmin - 2 * x)[None, :].expand(sp.ny, sp.nx)
    dfy = (sp.ymax + sp.ymin - 2 * y)[:, None].expand(sp.ny, sp.nx)
    inner = (slice(1, None), slice(1, None))
    assert torch.allclose(O.ddx(sp, fx)[inner], dfx[inner], atol=1e-12)
    assert torch.allclose(O.ddy(sp, fy)[inner], dfy[inner], atol=1e-12)
    # orientation: an x-only function has no y derivative away from the wall row
    assert float(O.ddy(sp, fx)[2:-1, 1:].abs().max()) < 1e-12
    assert torch.all(O.ddx(sp, fx)[:, 0] == 0) and torch.all(O.ddx(sp, fx)[0, :] == 0)


@pytest.mark.parametrize("nx,ny", [(16, 16), (24, 10), (64, 48)])
def test_fft_dst_matches_matrix_dst(nx, ny):
    """The O(n log n) DST-I (odd-extension FFT) reproduces the matrix definition."""
    sp = spec(nx=nx, ny=ny)
    a = torch.randn(ny, nx, generator=torch.Generator().manual_seed(nx * ny), dtype=torch.float64)
    ref = O.dst2(sp, a)
    with O.dst_algorithm("fft"):
        got = O.dst2(sp, a)
        f = O.poisson_solve(sp, a)
    assert float((got - ref).abs().max()) <= 1e-12 * float(ref.abs().max())
    assert float((f - O.poisson_solve(sp, a)).abs().max()) <= 1e-12 * float(f.abs().max())
    assert O.DST_ALGORITHM == "matrix"
