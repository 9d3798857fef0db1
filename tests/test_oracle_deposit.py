"""Pins for the oracle's shapes, deposition and gather (Sec. 3.2, orders 0-3 transverse).

The brute-force reference evaluates the centred cardinal B-spline from its
truncated-power closed form, a different formula from the oracle's local
"floor + polynomial pieces" weights.
"""
import math

import pytest
import torch

import oracle as O


def spec(nx=14, ny=12, order=1):
    return O.GridSpec(nx=nx, ny=ny, nzeta=4, xmin=-2.0, xmax=2.2, ymin=-1.5, ymax=1.5,
                      zeta_min=0.0, zeta_max=1.0, shape_order=order)


def bspline(t, p):
    """Centred cardinal B-spline of degree p via truncated powers."""
    if p == 0:
        return 1.0 if -0.5 <= t < 0.5 else 0.0
    s = 0.0
    for k in range(p + 2):
        v = t + (p + 1) / 2.0 - k
        if v > 0:
            s += (-1) ** k * math.comb(p + 1, k) * v ** p
    return s / math.factorial(p)


def rand_particles(sp, n, margin, seed):
    g = torch.Generator().manual_seed(seed)
    x = sp.xmin + (margin + (sp.nx - 2 * margin) * torch.rand(n, generator=g, dtype=torch.float64)) * sp.dx
    y = sp.ymin + (margin + (sp.ny - 2 * margin) * torch.rand(n, generator=g, dtype=torch.float64)) * sp.dy
    v = torch.randn(n, generator=g, dtype=torch.float64)
    return x, y, v


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_deposit_brute_force(order):
    sp = spec(nx=9, ny=8, order=order)
    x, y, v = rand_particles(sp, 40, 0.0, 11 + order)
    (got,) = O.deposit(sp, x, y, [v], order)
    ref = torch.zeros(sp.ny, sp.nx, dtype=torch.float64)
    for p in range(x.shape[0]):
        ux = (float(x[p]) - sp.xmin) / sp.dx
        uy = (float(y[p]) - sp.ymin) / sp.dy
        for i in range(1, sp.ny):
            for j in range(1, sp.nx):
                ref[i, j] += float(v[p]) * bspline(ux - j, order) * bspline(uy - i, order)
    assert torch.allclose(got, ref, atol=1e-13)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_charge_conservation(order):
    sp = spec(order=order)
    x, y, v = rand_particles(sp, 500, 2.5, 5 + order)  # >= 2.5 cells from the wall
    (rho,) = O.deposit(sp, x, y, [v], order)
    assert abs(float(rho.sum()) - float(v.sum())) <= 1e-13 * float(v.abs().sum())


@pytest.mark.parametrize("order", [0, 1, 2, 3])
@pytest.mark.parametrize("ppc", [(1, 1), (2, 1), (2, 2)])
def test_partition_of_unity(order, ppc):
    sp = spec(order=order)
    sp.ppc_x, sp.ppc_y = ppc
    st = O.plasma_init(sp)
    (n,) = O.deposit(sp, st["x"], st["y"], [st["w"] / (sp.dx * sp.dy)], order)
    inner = n[3:-3, 3:-3]
    assert torch.allclose(inner, torch.ones_like(inner), atol=1e-14)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_reproduces_affine(order):
    sp = spec(order=order)
    xs = sp.xmin + torch.arange(sp.nx, dtype=torch.float64) * sp.dx
    ys = sp.ymin + torch.arange(sp.ny, dtype=torch.float64) * sp.dy
    F = 0.3 + 1.7 * xs[None, :] - 0.9 * ys[:, None]
    x, y, _ = rand_particles(sp, 300, 2.5, 21)
    (g,) = O.gather(sp, x, y, [F], order)
    assert torch.allclose(g, 0.3 + 1.7 * x - 0.9 * y, atol=1e-12)


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_gather_is_deposit_transpose(order):
    sp = spec(order=order)
    x, y, w = rand_particles(sp, 200, 0.0, 31)  # includes particles touching the wall
    g = torch.Generator().manual_seed(9)
    F = torch.randn(sp.ny, sp.nx, generator=g, dtype=torch.float64)
    (D,) = O.deposit(sp, x, y, [w], order)
    (G,) = O.gather(sp, x, y, [F], order)
    lhs, rhs = float((F * D).sum()), float((w * G).sum())
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


def test_rho_minus_jz_identity():
    sp = spec(order=2)
    x, y, _ = rand_particles(sp, 300, 1.0, 41)
    g = torch.Generator().manual_seed(4)
    st = dict(x=x, y=y, ux=0.3 * torch.randn(300, generator=g, dtype=torch.float64),
              uy=0.3 * torch.randn(300, generator=g, dtype=torch.float64),
              psi=0.5 * torch.rand(300, generator=g, dtype=torch.float64) - 0.4,
              w=torch.rand(300, generator=g, dtype=torch.float64),
              alive=torch.ones(300, dtype=torch.bool))
    rho, jx, jy, jz, chi = O.plasma_deposit_full(sp, st)
    (ref,) = O.deposit(sp, x, y, [O.PLASMA_Q * st["w"] / (sp.dx * sp.dy)], 2)
    assert torch.allclose(rho - jz, ref, atol=1e-13)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_fp32_weight_knob(order):
    """The single-precision weight knob (a rounding-floor probe): each weight is the
    FP32 rounding of the brute-force B-spline value to within a few FP32 ulps, the
    weights still sum to one to FP32 precision, and the default FP64 path is unchanged
    by the knob's existence (it matches the brute force to 1e-14)."""
    g = torch.Generator().manual_seed(11 + order)
    u = 3.0 + 20.0 * torch.rand(400, generator=g, dtype=torch.float64)
    for wdt, tol in ((torch.float64, 1e-14), (torch.float32, 4e-7)):
        j0, w = O.qsa.shape_1d(u, order, wdt)
        assert all(t.dtype == torch.float64 for t in w)
        s = sum(w)
        assert float((s - 1.0).abs().max()) <= (1e-14 if wdt == torch.float64 else 4e-7)
        for a, wa in enumerate(w):
            ref = torch.tensor([bspline(float(uu) - float(j0[i] + a), order) for i, uu in enumerate(u)],
                               dtype=torch.float64)
            assert float((wa - ref).abs().max()) <= tol, (wdt, a)
    # FP32 weights are not the FP64 ones (the knob does something), but are close
    _, w64 = O.qsa.shape_1d(u, order, torch.float64)
    _, w32 = O.qsa.shape_1d(u, order, torch.float32)
    d = max(float((a - b).abs().max()) for a, b in zip(w32, w64))
    assert 0.0 < d <= 4e-7


@pytest.mark.parametrize("order", [1, 2, 3])
def test_chi_of_the_unperturbed_plasma_is_the_explicit_shift(order):
    """chi = sum q^2 w S g / (M A): a plasma at rest in its initial placement (g = 1) deposits the
    density times q^2/M on every node away from the walls (the lattice's partition of unity), the
    value explicit_shift computes from the grid parameters alone."""
    sp = O.GridSpec(nx=24, ny=20, nzeta=2, xmin=-3.0, xmax=3.0, ymin=-2.5, ymax=2.5, zeta_min=0.0, zeta_max=1.0,
                    shape_order=order, ppc_x=2, ppc_y=1, n0_scale=1.3)
    st = O.plasma_init(sp)
    *_, chi = O.plasma_deposit_full(sp, st)
    interior = chi[3:-3, 3:-3]
    assert float((interior - O.explicit_shift(sp)).abs().max()) <= 1e-13
    assert O.explicit_shift(sp) == pytest.approx(1.3)


def test_chi_over_rho_is_q_over_m_gamma_per_particle():
    """Per particle, chi / rho = (q^2 g / M) / (q gamma g) = q / (M gamma), node by node."""
    sp = spec(order=2)
    g = torch.Generator().manual_seed(9)
    for _ in range(3):
        x, y, _ = rand_particles(sp, 1, 2.0, int(torch.randint(0, 1000, (1,), generator=g)))
        st = dict(x=x, y=y, ux=0.4 * torch.randn(1, generator=g, dtype=torch.float64),
                  uy=0.4 * torch.randn(1, generator=g, dtype=torch.float64),
                  psi=torch.tensor([-0.3], dtype=torch.float64), w=torch.tensor([0.7], dtype=torch.float64),
                  alive=torch.ones(1, dtype=torch.bool))
        rho, _, _, _, chi = O.plasma_deposit_full(sp, st)
        gam = float(O.gamma_of(st["ux"], st["uy"], st["psi"]))
        nz = rho.abs() > 1e-12
        ratio = chi[nz] / rho[nz]
        assert torch.allclose(ratio, torch.full_like(ratio, O.PLASMA_Q / (O.PLASMA_M * gam)), rtol=1e-13, atol=0)


def test_trial_jperp_is_the_full_deposit_of_the_valid_particles():
    """The predictor-corrector's J_perp deposit of trial particles equals the J_perp of the full
    deposit over the same particles, and particles flagged invalid (here with non-finite states)
    contribute nothing."""
    sp = spec(order=3)
    x, y, _ = rand_particles(sp, 200, 1.5, 77)
    g = torch.Generator().manual_seed(5)
    ux = 0.5 * torch.randn(200, generator=g, dtype=torch.float64)
    uy = 0.5 * torch.randn(200, generator=g, dtype=torch.float64)
    psi = 0.6 * torch.rand(200, generator=g, dtype=torch.float64) - 0.5
    w = torch.rand(200, generator=g, dtype=torch.float64)
    ok = torch.rand(200, generator=g) > 0.3
    xb, psib = x.clone(), psi.clone()
    xb[~ok] = float("nan")
    psib[~ok] = float("inf")
    jx, jy = O.plasma_deposit_jperp(sp, xb, y, ux, uy, psib, w, ok)
    st = dict(x=x, y=y, ux=ux, uy=uy, psi=psi, w=w, alive=ok)
    _, fx, fy, _, _ = O.plasma_deposit_full(sp, st)
    assert torch.isfinite(jx).all() and torch.isfinite(jy).all()
    assert torch.allclose(jx, fx, rtol=0, atol=1e-13) and torch.allclose(jy, fy, rtol=0, atol=1e-13)
