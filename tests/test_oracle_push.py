"""Pins for the oracle's plasma push (Sec. 3.2, Eqs. for x_perp, u_perp, Psi; AB5) and beam push.

derivs is checked against the Lorentz force re-parametrised by zeta (an
independent formulation with full E and B vectors and cross products); the
Psi equation against the invariant Psi_p - psi(x_p) for fields derived from a
potential; AB5 against exact integration of quartics and its convergence order.
"""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp

import oracle as O


def T(v):
    return torch.tensor(v, dtype=torch.float64)


def lorentz_zeta(qm, ux, uy, psi, E, B):
    """du/dzeta from du/dt = (q/M)(E + v x B) and dzeta/dt = v_z - 1 (c = 1)."""
    opp = 1.0 + psi
    gam = (1.0 + ux * ux + uy * uy + opp * opp) / (2.0 * opp)
    uz = gam - opp  # gamma - u_z = 1 + Psi
    v = np.array([ux, uy, uz]) / gam
    F = qm * (np.asarray(E) + np.cross(v, B))
    dzdt = v[2] - 1.0
    dxdz = v[:2] / dzdt
    dudz = F / dzdt
    # d(gamma - u_z)/dt = (q/M)(E.v - F_z/(q/M)) ; Psi = gamma - u_z - 1
    dpsi = (qm * np.dot(E, v) - F[2]) / dzdt
    return np.array([dxdz[0], dxdz[1], dudz[0], dudz[1], dpsi])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("qm", [-1.0, 1.0 / 1836.0, -2.0])
def test_derivs_match_lorentz_force(seed, qm):
    rng = np.random.default_rng(seed)
    ux, uy = rng.normal(scale=0.7, size=2)
    psi = rng.uniform(-0.7, 1.5)
    E = rng.normal(size=3)
    B = rng.normal(size=3)
    F = (E[0] - B[1], E[1] + B[0], E[2], B[0], B[1], B[2])  # (ExmBy, EypBx, Ez, Bx, By, Bz)
    got = np.array([float(v) for v in O.derivs(qm, T(ux), T(uy), T(psi), [T(f) for f in F])])
    ref = lorentz_zeta(qm, ux, uy, psi, E, B)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_psi_tracks_potential():
    """With ExmBy, EypBx, Ez = -grad(psi), Psi_p - psi(x_p(zeta), zeta) is constant for any B."""
    def pot(x, y, z):
        return 0.3 * math.sin(x + 0.2 * z) * math.cos(0.7 * y) + 0.1 * z * x

    def grad(x, y, z):
        ex = 0.3 * math.cos(x + 0.2 * z) * math.cos(0.7 * y) + 0.1 * z
        ey = -0.21 * math.sin(x + 0.2 * z) * math.sin(0.7 * y)
        ez = 0.06 * math.cos(x + 0.2 * z) * math.cos(0.7 * y) + 0.1 * x
        return ex, ey, ez

    def rhs(z, s):
        x, y, ux, uy, psi = s
        gx, gy, gz = grad(x, y, z)
        F = [T(v) for v in (-gx, -gy, -gz, 0.4 * math.sin(z), -0.3, 0.25 * x)]
        d = O.derivs(-1.0, T(ux), T(uy), T(psi), F)
        return [float(v) for v in d]

    s0 = [0.2, -0.1, 0.05, 0.0, pot(0.2, -0.1, 0.0)]
    sol = solve_ivp(rhs, (0.0, -6.0), s0, rtol=1e-11, atol=1e-12, dense_output=True)
    inv = [sol.y[4, k] - pot(sol.y[0, k], sol.y[1, k], sol.t[k]) for k in range(sol.t.size)]
    assert max(abs(v - inv[0]) for v in inv) < 1e-8


def ab5_integrate(fun, y0, z0, dz, nsteps):
    """March y' = fun(z) (vector) backwards in zeta with AB5 from exact history."""
    hist = [[T(fun(z0 + k * dz))] for k in range(0, 5)]  # f_i, f_{i-1}, ..
    y = [T(y0)]
    z = z0
    for _ in range(nsteps):
        y = O.ab5_step(y, hist, dz)
        z -= dz
        hist = [[T(fun(z))]] + hist[:4]
    return float(y[0]), z


def test_ab5_exact_on_quartic():
    c = (0.3, -1.1, 0.7, 0.25, -0.05)
    P = lambda z: sum(ck * z ** k for k, ck in enumerate(c))  # noqa: E731
    Q = lambda z: sum(ck * z ** (k + 1) / (k + 1) for k, ck in enumerate(c))  # noqa: E731
    y0, z0, dz = 1.3, 0.4, 0.17
    y, z = ab5_integrate(P, Q(z0) + y0, z0, dz, 7)
    assert abs(y - (Q(z) + y0)) < 1e-12


def test_ab5_fifth_order():
    errs = []
    for n in (20, 40, 80):
        dz = 1.5 / n  # interval [-0.5, 1]: the leading error term does not cancel
        y, z = ab5_integrate(math.cos, math.sin(1.0), 1.0, dz, n)
        errs.append(abs(y - math.sin(z)))
    order = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(4.6 < o < 5.4 for o in order), order


def test_constant_ez_gives_linear_psi():
    F = [T(v) for v in (0.0, 0.0, 0.37, 0.0, 0.0, 0.0)]
    d = O.derivs(-1.0, T(0.0), T(0.0), T(0.2), F)
    assert float(d[4]) == pytest.approx(-0.37, abs=1e-15)
    assert float(d[0]) == 0.0 and float(d[2]) == 0.0


# ---------------------------------------------------------------- beam push pins

def beam_spec():
    return O.GridSpec(nx=32, ny=32, nzeta=8, xmin=-4.0, xmax=4.0, ymin=-4.0, ymax=4.0,
                      zeta_min=-2.0, zeta_max=2.0, shape_order=2)


def uniform_fields(sp, vals):
    out = []
    for v in vals:
        f = torch.full((sp.ny, sp.nx), float(v), dtype=torch.float64)
        out.append(f)
    return out


def small_beam(n=50, seed=0, gamma=200.0):
    rng = np.random.default_rng(seed)
    return O.as_beam(dict(x=rng.normal(scale=0.3, size=n), y=rng.normal(scale=0.3, size=n),
                          zeta=rng.uniform(-1, 1, size=n), ux=rng.normal(size=n), uy=rng.normal(size=n),
                          uz=np.full(n, gamma), w=np.ones(n)))


def test_beam_push_pure_bz_gyrates():
    sp = beam_spec()
    b = small_beam()
    sel = torch.arange(50)
    F = uniform_fields(sp, (0.0, 0.0, 0.0, 0.0, 0.0, 0.8))
    nb = O.beam_push(sp, b, sel, F, dt=3.0)
    u0 = torch.sqrt(b["ux"] ** 2 + b["uy"] ** 2)
    u1 = torch.sqrt(nb["ux"] ** 2 + nb["uy"] ** 2)
    assert torch.allclose(u0, u1, rtol=1e-13)
    assert torch.allclose(nb["uz"], b["uz"], rtol=1e-14)
    # d(phi)/dt = -(q/M) Bz / gamma; the Boris step turns u by -2 atan((q/M) Bz dt / (2 gamma))
    gam = torch.sqrt(1 + b["ux"] ** 2 + b["uy"] ** 2 + b["uz"] ** 2)
    ang = torch.atan2(nb["uy"], nb["ux"]) - torch.atan2(b["uy"], b["ux"])
    ang = torch.remainder(ang + math.pi, 2 * math.pi) - math.pi
    expect = -2 * torch.atan(-1.0 * 0.8 * 3.0 / (2 * gam))
    assert torch.allclose(ang, expect, atol=1e-12)


def test_beam_push_pure_ez_kick():
    sp = beam_spec()
    b = small_beam()
    sel = torch.arange(50)
    F = uniform_fields(sp, (0.0, 0.0, 0.05, 0.0, 0.0, 0.0))
    nb = O.beam_push(sp, b, sel, F, dt=2.0)
    assert torch.allclose(nb["uz"] - b["uz"], torch.full_like(b["uz"], -1.0 * 0.05 * 2.0), atol=1e-12)


def test_beam_push_time_reversible():
    sp = beam_spec()
    g = torch.Generator().manual_seed(1)
    F = [0.05 * torch.randn(sp.ny, sp.nx, generator=g, dtype=torch.float64) for _ in range(6)]
    b = small_beam(seed=3)
    sel = torch.arange(50)
    fwd = O.beam_push(sp, b, sel, F, dt=1.5)
    back = O.beam_push(sp, fwd, sel, F, dt=-1.5)
    for k in ("x", "y", "zeta", "ux", "uy", "uz"):
        assert torch.allclose(back[k], b[k], atol=1e-11), k
