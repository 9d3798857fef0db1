"""Plain FP64 restatement of the quasi-static PIC slice loop of arXiv:2109.10277.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Units are the paper's normalized units (Sec. 6): lengths in 1/k_p, fields in
E0 = m c omega_p / e, densities in n0, c = eps0 = mu0 = 1.  Plasma electrons have
q = -1, M = 1; ions are immobile.

Everything is written with differentiable torch ops on CPU float64, so running
``sweep`` under autograd gives the oracle's taped adjoint.

Readings of the paper (it is silent or only cites a reference on these points):
  * grid: nodes x_j = xmin + j dx, j = 0..nx; nodes 0 and nx lie on the Dirichlet
    wall and are zero.  Arrays are (ny, nx) over nodes 0..n-1 with row/col 0 zero.
    The interior is transformed by the DST-I of Sec. 3.2 (fast Poisson solver),
    i.e. S_jk = sin(pi j k / n); the 5-point Laplacian is the operator DST-I
    diagonalises exactly.
  * transverse derivatives are second-order central differences on interior
    nodes; d(J_perp)/d(zeta) is central between slices zeta+dzeta and zeta-dzeta
    (Sec. 3.2, predictor-corrector).
  * shapes are cardinal B-splines of order 0-3 (Sec. 3.2 deposition), used for
    both gather and deposit; weight landing outside nodes 1..n-1 is discarded
    (deposit) or reads zero (gather).
  * a macroparticle represents a fixed flux, so its density is w*gamma/((1+Psi)A);
    with gamma - u_z = 1 + Psi (Eq. for gamma_p) this gives rho - J_z = q w S / A.
  * chi = q^2 w S / (M (1+Psi) A) (the explicit solver's susceptibility; output only).
  * ions: minus the electron charge deposited once from the initial positions.
  * predictor-corrector: guess B(i) = 2 B(i-1) - B(i-2) (B = 0 before the box),
    fixed n_pc iterations with mixing weight pc_mix, no early exit.
  * a particle is removed (weight to zero, state frozen) when after a full step
    1 + Psi < psi_guard, it leaves the open box, or a value is not finite; a trial
    state failing the same test is skipped in the trial deposit.
  * beam push: drift-kick-drift with a Boris kick (second order, time
    reversible), fields of the particle's own slice (order-0 longitudinal).
"""
from __future__ import annotations

import contextlib
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

DT = torch.float64
DEV = torch.device("cpu")


@contextlib.contextmanager
def working_precision(dtype: torch.dtype):
    """Evaluate the oracle in another floating-point type inside the block.

    The method is FP64 (the default).  ``working_precision(torch.float32)`` runs the
    same steps with every tensor in single precision: a test knob that measures the
    single-precision rounding floor of the algorithm, the reference point for a
    mixed-precision implementation's error.  Not re-entrant across threads.
    A test knob (no passage of the paper): the same steps in another float type."""
    global DT
    old = DT
    DT = dtype
    try:
        yield
    finally:
        DT = old

# Fifth-order Adams-Bashforth weights (Sec. 3.2 plasma push): beta_k for f_{i-k}.
AB5 = (1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0)

FIELD_NAMES = ("rho", "jx", "jy", "jz", "chi", "psi", "exmby", "eypbx", "ez", "bx", "by", "bz")


@dataclass(frozen=True)
class Species:
    """One plasma species (Sec. 6 feature list: plasmas of several species and profiles, ion
    motion).  charge and mass in units of e and m_e; the push uses q/M (Sec. 3.2 plasma
    equations), the deposits q and q^2/M.  neutralize: an immobile background of the opposite
    charge sits at the species' initial positions (the default electron plasma's ions);
    without it the species' own initial charge is left in the slice."""
    charge: float = -1.0
    mass: float = 1.0
    n0_scale: float = 1.0
    ppc_x: int = 1
    ppc_y: int = 1
    radial_profile: Optional[Sequence[float]] = None
    profile_rmax: float = 0.0
    neutralize: bool = True


@dataclass
class GridSpec:
    """Transverse Dirichlet box, zeta range and plasma/solver parameters (Sec. 2, 3.2)."""
    nx: int
    ny: int
    nzeta: int
    xmin: float
    xmax: float
    ymin: float
    ymax: float
    zeta_min: float
    zeta_max: float
    shape_order: int = 1
    ppc_x: int = 1
    ppc_y: int = 1
    radial_profile: Optional[Sequence[float]] = None
    profile_rmax: float = 0.0
    n0_scale: float = 1.0
    n_pc_iter: int = 5          # predictor-corrector iterations, or the explicit solver's PCG iterations
    pc_mix: float = 0.05
    psi_guard: float = 0.02
    bperp_solver: str = "pc"    # "pc": predictor-corrector; "explicit": Helmholtz-like equation in chi
    # plasma species; empty: one electron species (q = -1, M = 1) with immobile ions, placed by
    # ppc_x, ppc_y, radial_profile, profile_rmax and n0_scale above
    species: Sequence[Species] = ()
    # "float32": B-spline weights formed from an FP32 cell fraction in FP32 arithmetic
    # (then widened).  A test knob that measures the rounding floor of a single-precision
    # deposit/gather; the method itself is the default, FP64.
    weight_dtype: str = "float64"

    @property
    def dx(self) -> float:
        """Cell size in x (nx cells between the walls)."""
        return (self.xmax - self.xmin) / self.nx

    @property
    def dy(self) -> float:
        """Cell size in y."""
        return (self.ymax - self.ymin) / self.ny

    @property
    def dzeta(self) -> float:
        """Slice thickness (Sec. 2: the box is cut into nzeta transverse slices)."""
        return (self.zeta_max - self.zeta_min) / self.nzeta


# ----------------------------------------------------------------------------
# Fast Poisson solver (Sec. 3.2: DST-I, Dirichlet boundary)
# ----------------------------------------------------------------------------

def dst_matrix(n: int) -> torch.Tensor:
    """S_jk = sin(pi j k / n), j, k = 0..n-1 (row/col 0 are zero): DST-I with a zero border.
    Sec. 3.2 (Poisson solver by a DST of the first type, read as acting on the interior nodes with
    the wall nodes zero)."""
    j = torch.arange(n, dtype=torch.int64)
    m = torch.remainder(torch.outer(j, j), 2 * n)  # exact argument reduction
    return torch.sin(math.pi * m.to(DT) / n)


def laplace_eigs(spec: GridSpec) -> torch.Tensor:
    """Eigenvalues lambda[l, k] of the 5-point Laplacian for DST-I mode (k in x, l in y).
    Sec. 3.2 and Eq. psi: the 5-point Laplacian is the operator the DST-I diagonalises (a reading:
    the paper does not name the discrete Laplacian)."""
    k = torch.arange(spec.nx, dtype=DT)
    l = torch.arange(spec.ny, dtype=DT)
    ex = -(4.0 / spec.dx ** 2) * torch.sin(math.pi * k / (2 * spec.nx)) ** 2
    ey = -(4.0 / spec.dy ** 2) * torch.sin(math.pi * l / (2 * spec.ny)) ** 2
    return ey[:, None] + ex[None, :]


DST_ALGORITHM = "matrix"


@contextlib.contextmanager
def dst_algorithm(name: str):
    """Choose how dst2 evaluates the DST-I inside the block: "matrix" (the default, the
    transform's definition as a product with S) or "fft" (the same sums in O(n log n) per
    row, through the FFT of the odd extension).  The two differ only in rounding order:
    the FFT form serves the timed CPU baseline and measures how much the sweep amplifies
    the DST's own rounding.  Not re-entrant across threads.
    A test knob: the same DST-I of Sec. 3.2 evaluated another way."""
    global DST_ALGORITHM
    old = DST_ALGORITHM
    if name not in ("matrix", "fft"):
        raise ValueError(name)
    DST_ALGORITHM = name
    try:
        yield
    finally:
        DST_ALGORITHM = old


def dst1_rows_fft(a: torch.Tensor) -> torch.Tensor:
    """b_k = sum_{j=1}^{n-1} a_j sin(pi j k / n) along the last axis (node 0 on the wall).

    The odd extension e = (a_0 .. a_{n-1}, 0, -a_{n-1} .. -a_1) of length 2n has the discrete
    Fourier transform sum_j a_j (e^{-i pi j k/n} - e^{i pi j k/n}) = -2i sum_j a_j sin(pi j k/n)
    (a_0 only adds a real constant), so b_k = -Im(E_k) / 2.  Sec. 3.2 (the DST-I by FFTs)."""
    n = a.shape[-1]
    ext = torch.cat([a, torch.zeros_like(a[..., :1]), -a[..., 1:].flip(-1)], dim=-1)
    return -0.5 * torch.fft.rfft(ext, dim=-1)[..., :n].imag


def dst2(spec: GridSpec, a: torch.Tensor) -> torch.Tensor:
    """Unnormalised 2D DST-I of the interior: S_y a S_x.  Sec. 3.2 (DST-I)."""
    if DST_ALGORITHM == "fft":
        t = dst1_rows_fft(a)                                        # a S_x: along x
        return dst1_rows_fft(t.transpose(-1, -2)).transpose(-1, -2)  # S_y (.): along y
    return dst_matrix(spec.ny) @ a @ dst_matrix(spec.nx)


def poisson_solve(spec: GridSpec, s: torch.Tensor) -> torch.Tensor:
    """f = L^{-1} s with L the 5-point Laplacian and f = 0 on the wall (Sec. 3.2).

    f_hat = (S_y s S_x) / lambda;  f = (2/nx)(2/ny) S_y f_hat S_x.
    """
    lam = laplace_eigs(spec)
    inv = torch.zeros_like(lam)
    inv[1:, 1:] = 1.0 / lam[1:, 1:]
    f_hat = dst2(spec, s) * inv
    return (4.0 / (spec.nx * spec.ny)) * dst2(spec, f_hat)


def _wall_mask(spec: GridSpec) -> torch.Tensor:
    m = torch.ones(spec.ny, spec.nx, dtype=DT)
    m[0, :] = 0.0
    m[:, 0] = 0.0
    return m


def ddx(spec: GridSpec, f: torch.Tensor) -> torch.Tensor:
    """Central x-derivative on interior nodes; node nx (wall) reads 0, wall outputs are 0.
    The transverse derivatives of Eqs. exmby, ez, bz and bxby (central differences: a reading, the
    paper does not name the stencil)."""
    fp = torch.cat([f, torch.zeros_like(f[..., :1])], dim=-1)  # columns 0..nx
    d = torch.zeros_like(f)
    d = torch.cat([d[..., :1], (fp[..., 2:] - fp[..., :-2]) / (2.0 * spec.dx)], dim=-1)
    return d * _wall_mask(spec)


def ddy(spec: GridSpec, f: torch.Tensor) -> torch.Tensor:
    """Central y-derivative on interior nodes; node ny (wall) reads 0, wall outputs are 0.
    The transverse derivatives of Eqs. exmby, ez, bz and bxby (central differences: a reading, the
    paper does not name the stencil)."""
    fp = torch.cat([f, torch.zeros_like(f[..., :1, :])], dim=-2)
    d = torch.cat([torch.zeros_like(f[..., :1, :]), (fp[..., 2:, :] - fp[..., :-2, :]) / (2.0 * spec.dy)], dim=-2)
    return d * _wall_mask(spec)


def laplacian(spec: GridSpec, f: torch.Tensor) -> torch.Tensor:
    """The 5-point Laplacian on interior nodes (wall nodes read 0; wall outputs are 0): the
    operator poisson_solve inverts.  Eq. psi (the 5-point operator, a reading)."""
    fp = torch.nn.functional.pad(f, (0, 1, 0, 1))             # nodes nx, ny (wall) = 0
    c = fp[1:-1, 1:-1]
    lap = torch.zeros_like(f)
    lap[1:, 1:] = ((fp[1:-1, 2:] - 2.0 * c + fp[1:-1, :-2]) / spec.dx ** 2 +
                   (fp[2:, 1:-1] - 2.0 * c + fp[:-2, 1:-1]) / spec.dy ** 2)
    return lap


def shifted_solve(spec: GridSpec, s: torch.Tensor, c: float) -> torch.Tensor:
    """f = (L - c)^{-1} s for a constant c >= 0 (DST-I with 1/(lambda - c); f = 0 on the wall).
    Sec. 3.2 (explicit field solver; its equation read from Ampere's law with the plasma's
    d/dzeta J_perp from the particle equations, the paper citing it without printing it)."""
    lam = laplace_eigs(spec)
    inv = torch.zeros_like(lam)
    inv[1:, 1:] = 1.0 / (lam[1:, 1:] - c)
    return (4.0 / (spec.nx * spec.ny)) * dst2(spec, dst2(spec, s) * inv)


def explicit_shift(spec: GridSpec) -> float:
    """The explicit solver's preconditioner shift c: the unperturbed chi, sum q^2 n0 / M over the
    plasma species (n0_scale for the default electrons).  Sec. 3.2 (explicit field solver; its equation read from Ampere's law with the plasma's
    d/dzeta J_perp from the particle equations, the paper citing it without printing it)."""
    if not spec.species:
        return spec.n0_scale
    return sum(s.charge * s.charge * s.n0_scale / s.mass for s in spec.species)


def helmholtz_pcg(spec: GridSpec, chi: torch.Tensor, rhs: Sequence[torch.Tensor], x0: Sequence[torch.Tensor],
                  c: float, iters: int):
    """Solve (L - chi) B = rhs for each right-hand side: preconditioned conjugate gradients on
    the symmetric positive definite form (chi - L) B = -rhs, preconditioner (c - L)^{-1} (one
    shifted DST-I solve), start x0, a fixed number of iterations `iters` (no early exit; a
    zero residual stops the update).  Returns the iterates and the final relative residuals.
    Sec. 3.2 (explicit field solver: the Helmholtz-like equation, read from Ampere's law with the
    plasma's d/dzeta J_perp from the particle equations)."""
    mask = _wall_mask(spec)
    A = lambda v: chi * v * mask - laplacian(spec, v)  # noqa: E731
    P = lambda v: -shifted_solve(spec, v, c)  # noqa: E731
    out, resid = [], []
    for b_, x in zip(rhs, x0):
        b = -b_ * mask
        x = x * mask
        r = b - A(x)
        z = P(r)
        p = z
        rz = (r * z).sum()
        for k in range(iters):
            q = A(p)
            pq = (p * q).sum()
            alpha = torch.where(pq != 0, rz / torch.where(pq != 0, pq, torch.ones_like(pq)), torch.zeros_like(pq))
            x = x + alpha * p
            r = r - alpha * q
            if k < iters - 1:
                z = P(r)
                rz_new = (r * z).sum()
                beta = torch.where(rz != 0, rz_new / torch.where(rz != 0, rz, torch.ones_like(rz)), torch.zeros_like(rz))
                p = z + beta * p
                rz = rz_new
        nb = float(torch.linalg.norm(b))
        resid.append(float(torch.linalg.norm(b - A(x))) / nb if nb > 0 else 0.0)
        out.append(x)
    return out, resid


# ----------------------------------------------------------------------------
# Shapes, deposition and gather (Sec. 3.2: order 0 longitudinal, 0-3 transverse)
# ----------------------------------------------------------------------------

def shape_1d(u: torch.Tensor, order: int, wdtype: torch.dtype = torch.float64):
    """B-spline weights of order `order` at node coordinate u (nodes at integers).

    Returns (j0, [w_0..w_p]): node j0 + a carries weight w_a.  The cell fraction and
    the weights are formed in `wdtype` (FP64 unless a rounding floor is being measured).
    Sec. 3.2 (deposition of orders 0-3 transversely; the same B-spline for gather and deposit, a
    reading).
    """
    def back(ws):
        """The weights in the coordinate's float type."""
        return [w.to(u.dtype) for w in ws]
    if order == 0:
        j0 = torch.floor(u + 0.5)
        return j0.to(torch.int64), [torch.ones_like(u)]
    if order == 1:
        j0 = torch.floor(u)
        d = (u - j0).to(wdtype)
        return j0.to(torch.int64), back([1.0 - d, d])
    if order == 2:
        jc = torch.floor(u + 0.5)
        d = (u - jc).to(wdtype)
        return (jc - 1).to(torch.int64), back([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2])
    if order == 3:
        jf = torch.floor(u)
        d = (u - jf).to(wdtype)
        return (jf - 1).to(torch.int64), back([
            (1.0 - d) ** 3 / 6.0,
            (4.0 - 6.0 * d * d + 3.0 * d ** 3) / 6.0,
            (1.0 + 3.0 * d + 3.0 * d * d - 3.0 * d ** 3) / 6.0,
            d ** 3 / 6.0,
        ])
    raise ValueError("shape order must be 0..3")


def _stencil(spec: GridSpec, x: torch.Tensor, y: torch.Tensor, order: int):
    """Yield (flat node index, weight) for every stencil node; invalid nodes get weight 0."""
    wdt = torch.float32 if spec.weight_dtype == "float32" else torch.float64
    jx0, wx = shape_1d((x - spec.xmin) / spec.dx, order, wdt)
    jy0, wy = shape_1d((y - spec.ymin) / spec.dy, order, wdt)
    for b in range(order + 1):
        jy = jy0 + b
        vy = (jy >= 1) & (jy <= spec.ny - 1)
        for a in range(order + 1):
            jx = jx0 + a
            valid = vy & (jx >= 1) & (jx <= spec.nx - 1)
            idx = torch.where(valid, jy * spec.nx + jx, torch.zeros_like(jx))
            yield idx, torch.where(valid, wx[a] * wy[b], torch.zeros_like(wx[a]))


def deposit(spec: GridSpec, x, y, values: Sequence[torch.Tensor], order: int, reverse: bool = False):
    """Scatter per-particle `values` onto the node grid with shape `order`.

    reverse=True visits the stencil offsets in the opposite order (the same sums,
    added in another order).  Sec. 3.2 (current deposition)."""
    outs = [torch.zeros(spec.ny * spec.nx, dtype=DT) for _ in values]
    stencil = list(_stencil(spec, x, y, order))
    for idx, wgt in (stencil[::-1] if reverse else stencil):
        outs = [o.index_add(0, idx, wgt * v) for o, v in zip(outs, values)]
    return [o.reshape(spec.ny, spec.nx) for o in outs]


def gather(spec: GridSpec, x, y, fields: Sequence[torch.Tensor], order: int):
    """Interpolate node `fields` to particle positions with shape `order`.
    Sec. 3.2 (field gather)."""
    flat = [f.reshape(-1) for f in fields]
    outs = [torch.zeros_like(x) for _ in fields]
    for idx, wgt in _stencil(spec, x, y, order):
        outs = [o + wgt * f[idx] for o, f in zip(outs, flat)]
    return outs


# ----------------------------------------------------------------------------
# Plasma push (Sec. 3.2, Eqs. for d(x_perp)/d(zeta), d(u_perp)/d(zeta), d(Psi)/d(zeta))
# ----------------------------------------------------------------------------

def derivs(q_over_m: float, ux, uy, psi, F):
    """zeta-derivatives (dx, dy, dux, duy, dpsi) of a plasma particle.

    F = (ExmBy, EypBx, Ez, Bx, By, Bz) gathered at the particle; q/M in units e/m_e.
    Sec. 3.2, Eq. 1 (the plasma particle equations).
    """
    exmby, eypbx, ez, bx, by, bz = F
    opp = 1.0 + psi
    g = 1.0 / opp
    gam = (1.0 + ux * ux + uy * uy + opp * opp) * 0.5 * g
    dxz = -ux * g
    dyz = -uy * g
    dux = -q_over_m * (gam * g * exmby + by + bz * g * uy)
    duy = -q_over_m * (gam * g * eypbx - bx - bz * g * ux)
    dpsi = -q_over_m * (g * (ux * exmby + uy * eypbx) - ez)
    return (dxz, dyz, dux, duy, dpsi)


def ab5_step(y: Sequence[torch.Tensor], fs: Sequence[Sequence[torch.Tensor]], dzeta: float):
    """One step zeta -> zeta - dzeta: y - dzeta * sum_k beta_k f_{i-k}; fs = [f_i, f_{i-1}, ..].
    Sec. 3.2 (fifth-order Adams-Bashforth plasma pusher)."""
    out = []
    for c in range(len(y)):
        acc = AB5[0] * fs[0][c]
        for k in range(1, 5):
            acc = acc + AB5[k] * fs[k][c]
        out.append(y[c] - dzeta * acc)
    return out


def gamma_of(ux, uy, psi):
    """Lorentz factor of a plasma particle, gamma_p = (1 + u_perp^2 + (1 + Psi)^2) / (2 (1 + Psi))
    (Sec. 3.2, the equation for gamma_p)."""
    opp = 1.0 + psi
    return (1.0 + ux * ux + uy * uy + opp * opp) / (2.0 * opp)


# ----------------------------------------------------------------------------
# Plasma state and deposits
# ----------------------------------------------------------------------------

PLASMA_Q = -1.0
PLASMA_M = 1.0


def plasma_species(spec: GridSpec) -> list:
    """The plasma species of a grid: spec.species, or the default electrons with immobile ions.
    Sec. 6 (plasmas of several species, ion motion), each pushed with its q/M (Sec. 3.2)."""
    if spec.species:
        return list(spec.species)
    return [Species(PLASMA_Q, PLASMA_M, spec.n0_scale, spec.ppc_x, spec.ppc_y, spec.radial_profile,
                    spec.profile_rmax, True)]


def plasma_init(spec: GridSpec, n0_scale: Optional[torch.Tensor] = None,
                radial_profile: Optional[torch.Tensor] = None, species: Optional[Species] = None):
    """ppc_x x ppc_y electrons per cell at sub-cell centres, at rest (Sec. 2); with `species`,
    that species' particles per cell, density scale and profile instead of the grid's.

    Ordering: cell row-major (iy, ix), then sub-particle (sy, sx).
    w = n0_scale * n(r) * dx * dy / ppc with n(r) linearly interpolated from the
    radial profile over [0, profile_rmax] (uniform if no profile).
    """
    if species is not None:
        spec = GridSpec(**{**spec.__dict__, "ppc_x": species.ppc_x, "ppc_y": species.ppc_y,
                           "radial_profile": species.radial_profile, "profile_rmax": species.profile_rmax,
                           "n0_scale": species.n0_scale, "species": ()})
    px, py = spec.ppc_x, spec.ppc_y
    iy, ix, sy, sx = torch.meshgrid(torch.arange(spec.ny), torch.arange(spec.nx),
                                    torch.arange(py), torch.arange(px), indexing="ij")
    x = spec.xmin + (ix.to(DT) + (sx.to(DT) + 0.5) / px) * spec.dx
    y = spec.ymin + (iy.to(DT) + (sy.to(DT) + 0.5) / py) * spec.dy
    x = x.reshape(-1)
    y = y.reshape(-1)
    if n0_scale is None:
        n0_scale = torch.tensor(spec.n0_scale, dtype=DT)
    dens = torch.ones_like(x)
    prof = radial_profile
    if prof is None and spec.radial_profile is not None:
        prof = torch.tensor(list(spec.radial_profile), dtype=DT)
    if prof is not None:
        npf = prof.shape[0]
        r = torch.sqrt(x * x + y * y)
        t = torch.clamp(r / spec.profile_rmax * (npf - 1), 0.0, float(npf - 1))
        k0 = torch.clamp(torch.floor(t).to(torch.int64), 0, npf - 2)
        fr = t - k0.to(DT)
        dens = prof[k0] * (1.0 - fr) + prof[k0 + 1] * fr
    w = n0_scale * dens * (spec.dx * spec.dy / (px * py))
    z = torch.zeros_like(x)
    return dict(x=x, y=y, ux=z.clone(), uy=z.clone(), psi=z.clone(), w=w,
                alive=torch.ones_like(x, dtype=torch.bool))


def plasma_deposit_full(spec: GridSpec, st, q=PLASMA_Q, m=PLASMA_M):
    """rho, Jx, Jy, Jz, chi of the plasma slice (Sec. 2 step 2; densities per reading above)."""
    A = spec.dx * spec.dy
    opp = 1.0 + st["psi"]
    g = 1.0 / opp
    gam = (1.0 + st["ux"] ** 2 + st["uy"] ** 2 + opp * opp) * 0.5 * g
    uz = (1.0 + st["ux"] ** 2 + st["uy"] ** 2 - opp * opp) * 0.5 * g
    qw = torch.where(st["alive"], q * st["w"], torch.zeros_like(st["w"])) / A
    vals = [qw * gam * g, qw * st["ux"] * g, qw * st["uy"] * g, qw * uz * g, qw * q * g / m]
    return deposit(spec, st["x"], st["y"], vals, spec.shape_order)


def explicit_sources(spec: GridSpec, st, F4, q=PLASMA_Q, m=PLASMA_M):
    """The plasma's d(J_perp)/d(zeta) at the current slice without its B_perp part (the
    explicit solver's source; reading: differentiate J_perp = sum q w S u_perp/((1+Psi) A) along
    zeta with the particle equations of Sec. 3.2).  F4 = (ExmBy, EypBx, Ez, Bz) gathered at the
    particles.  Returns the deposits (Fx, Fy, Jxx, Jxy, Jyy) with
      Fx = sum a S [g Gx - u_x g^2 Psi'],  Gx = -(q/M)(gamma g ExmBy + Bz g u_y),
      Fy = sum a S [g Gy - u_y g^2 Psi'],  Gy = -(q/M)(gamma g EypBx - Bz g u_x),
      Psi' = -(q/M)(g (u_x ExmBy + u_y EypBx) - Ez),  Jab = sum a S g^2 u_a u_b,
    a = q w / A, g = 1/(1+Psi); then d(Jx)/d(zeta) = Fx + dx Jxx + dy Jxy - (q/M) sum a S g By and
    d(Jy)/d(zeta) = Fy + dx Jxy + dy Jyy + (q/M) sum a S g Bx (the B terms are -chi By, chi Bx)."""
    A = spec.dx * spec.dy
    exmby, eypbx, ez, bz = F4
    ux, uy = st["ux"], st["uy"]
    opp = 1.0 + st["psi"]
    g = 1.0 / opp
    gam = (1.0 + ux * ux + uy * uy + opp * opp) * 0.5 * g
    qm = q / m
    a = torch.where(st["alive"], q * st["w"], torch.zeros_like(st["w"])) / A
    dpsi = -qm * (g * (ux * exmby + uy * eypbx) - ez)
    gx = -qm * (gam * g * exmby + bz * g * uy)
    gy = -qm * (gam * g * eypbx - bz * g * ux)
    g2 = g * g
    vals = [a * (g * gx - ux * g2 * dpsi), a * (g * gy - uy * g2 * dpsi),
            a * g2 * ux * ux, a * g2 * ux * uy, a * g2 * uy * uy]
    return deposit(spec, st["x"], st["y"], vals, spec.shape_order)


def _state_ok(spec: GridSpec, x, y, psi):
    fin = torch.isfinite(x) & torch.isfinite(y) & torch.isfinite(psi)
    inside = (x > spec.xmin) & (x < spec.xmax) & (y > spec.ymin) & (y < spec.ymax)
    return fin & inside & (1.0 + psi >= spec.psi_guard)


def plasma_deposit_jperp(spec: GridSpec, x, y, ux, uy, psi, w, ok, q=PLASMA_Q):
    """Jx, Jy of (trial) particles; particles with ok == False contribute nothing.
    Sec. 3.2 (predictor-corrector: J_perp of the trial particles; the macroparticle carries a fixed
    flux, n = w gamma / ((1 + Psi) A), a reading)."""
    A = spec.dx * spec.dy
    one = torch.ones_like(psi)
    safe = lambda t, fill: torch.where(ok, t, fill)  # noqa: E731
    xs, ys = safe(x, torch.full_like(x, spec.xmin)), safe(y, torch.full_like(y, spec.ymin))
    g = 1.0 / safe(1.0 + psi, one)
    qw = torch.where(ok, q * w, torch.zeros_like(w)) / A
    return deposit(spec, xs, ys, [qw * safe(ux, 0 * one) * g, qw * safe(uy, 0 * one) * g],
                   spec.shape_order)


def ion_background(spec: GridSpec, st0, q=PLASMA_Q, reverse: bool = False):
    """Immobile ions: minus the initial electron charge density, deposited with the same shape.
    Immobile ions (Sec. 4), read as minus the initial electron density deposited with the same shape."""
    A = spec.dx * spec.dy
    (rho_e,) = deposit(spec, st0["x"], st0["y"], [q * st0["w"] / A], spec.shape_order, reverse)
    return -rho_e


# ----------------------------------------------------------------------------
# Beams (Sec. 3.1: beam particles sorted per slice; order-0 longitudinal deposit)
# ----------------------------------------------------------------------------

def beam_bins(spec: GridSpec, zeta: torch.Tensor) -> torch.Tensor:
    """Slice index floor((zeta_max - zeta)/dzeta); -1 for particles outside [0, nzeta).
    Sec. 3.1 (beam particles sorted per slice), Sec. 3.2 (order 0 longitudinally)."""
    t = torch.floor((spec.zeta_max - zeta) / spec.dzeta)
    ok = torch.isfinite(t) & (t >= 0) & (t < spec.nzeta)
    return torch.where(ok, t, torch.full_like(t, -1.0)).to(torch.int64)


def beam_csr(spec: GridSpec, bins: torch.Tensor):
    """Counting-sort offsets: particles of slice i are order[off[i]:off[i+1]] (stable).
    Sec. 3.1 (beam particles sorted per slice)."""
    counts = torch.bincount(bins[bins >= 0], minlength=spec.nzeta)
    off = torch.zeros(spec.nzeta + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(counts, 0)
    sel = torch.nonzero(bins >= 0).reshape(-1)
    order = sel[torch.argsort(bins[sel], stable=True)]
    return off, order


def beam_deposit_slice(spec: GridSpec, beam, sel: torch.Tensor, channels=("rho", "jx", "jy", "jz")):
    """Beam rho, J of the particles `sel` (one slice): rho = q w S/(dx dy dzeta), J = rho u/gamma.
    Sec. 3.2 (deposition, order 0 longitudinally; the per-slice units a reading)."""
    x, y = beam["x"][sel], beam["y"][sel]
    ux, uy, uz, w = beam["ux"][sel], beam["uy"][sel], beam["uz"][sel], beam["w"][sel]
    gam = torch.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    r = beam["charge"] * w / (spec.dx * spec.dy * spec.dzeta)
    table = dict(rho=r, jx=r * ux / gam, jy=r * uy / gam, jz=r * uz / gam)
    return deposit(spec, x, y, [table[c] for c in channels], spec.shape_order)


def beam_push(spec: GridSpec, beam, sel, F, dt: float):
    """Drift-kick-drift (Boris kick) step of length dt for beam particles `sel`.

    F = slice fields (ExmBy, EypBx, Ez, Bx, By, Bz); E = (ExmBy + By, EypBx - Bx, Ez),
    B = (Bx, By, Bz).  zeta advances with v_z - 1.  Returns updated copies of the arrays.
    Sec. 3.2 (second-order symplectic beam integrator, read as drift-kick-drift with a Boris kick).
    """
    qm = beam["charge"] / beam["mass"]
    x, y, z = beam["x"][sel], beam["y"][sel], beam["zeta"][sel]
    ux, uy, uz = beam["ux"][sel], beam["uy"][sel], beam["uz"][sel]
    h = 0.5 * dt

    def drift(x, y, z, ux, uy, uz):
        """Half-step drift of the beam integrator (Sec. 3.2); zeta moves with v_z - 1."""
        ig = 1.0 / torch.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
        return x + h * ux * ig, y + h * uy * ig, z + h * (uz * ig - 1.0)

    x, y, z = drift(x, y, z, ux, uy, uz)
    exmby, eypbx, ez, bx, by, bz = gather(spec, x, y, F, spec.shape_order)
    ex, ey = exmby + by, eypbx - bx
    # Boris: half electric kick, magnetic rotation, half electric kick
    ux, uy, uz = ux + qm * h * ex, uy + qm * h * ey, uz + qm * h * ez
    ig = 1.0 / torch.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    tx, ty, tz = qm * h * bx * ig, qm * h * by * ig, qm * h * bz * ig
    s = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz)
    px = ux + (uy * tz - uz * ty)
    py = uy + (uz * tx - ux * tz)
    pz = uz + (ux * ty - uy * tx)
    ux = ux + s * (py * tz - pz * ty)
    uy = uy + s * (pz * tx - px * tz)
    uz = uz + s * (px * ty - py * tx)
    ux, uy, uz = ux + qm * h * ex, uy + qm * h * ey, uz + qm * h * ez
    x, y, z = drift(x, y, z, ux, uy, uz)
    out = dict(beam)
    for k, v in (("x", x), ("y", y), ("zeta", z), ("ux", ux), ("uy", uy), ("uz", uz)):
        out[k] = beam[k].index_copy(0, sel, v)
    return out


BEAM_MOMENT_NAMES = ("w", "x", "y", "ux", "uy", "xx", "yy", "uxux", "uyuy", "xux", "yuy")


def beam_moments(beam) -> torch.Tensor:
    """Weighted raw moments of a beam over all its particles (Sec. 6 precision study: the
    witness emittance): sum w, sum w x, sum w y, sum w ux, sum w uy, sum w x^2, sum w y^2,
    sum w ux^2, sum w uy^2, sum w x ux, sum w y uy."""
    w, x, y, ux, uy = (beam[k] for k in ("w", "x", "y", "ux", "uy"))
    return torch.stack([w.sum(), (w * x).sum(), (w * y).sum(), (w * ux).sum(), (w * uy).sum(),
                        (w * x * x).sum(), (w * y * y).sum(), (w * ux * ux).sum(), (w * uy * uy).sum(),
                        (w * x * ux).sum(), (w * y * uy).sum()])


def emittance(m) -> tuple:
    """Normalised rms emittances (eps_x, eps_y) from beam_moments: eps_x^2 = <dx^2><dux^2> - <dx dux>^2
    with centred, weight-averaged second moments (momenta in units of m c).
    Sec. 6 (the precision study's emittance; the definition a reading, the paper prints none)."""
    m = [float(v) for v in m]
    W = m[0]
    out = []
    for a, b, aa, bb, ab in ((1, 3, 5, 7, 9), (2, 4, 6, 8, 10)):
        ma, mb = m[a] / W, m[b] / W
        vaa = m[aa] / W - ma * ma
        vbb = m[bb] / W - mb * mb
        vab = m[ab] / W - ma * mb
        out.append(math.sqrt(max(vaa * vbb - vab * vab, 0.0)))
    return tuple(out)


def as_beam(arrays: dict, charge: float = -1.0, mass: float = 1.0):
    """Convert a dict of numpy/torch arrays (x, y, zeta, ux, uy, uz, w) to float64 tensors.
    Input marshalling (no passage of the paper)."""
    out = {k: torch.as_tensor(arrays[k], dtype=DT) for k in ("x", "y", "zeta", "ux", "uy", "uz", "w")}
    out["charge"] = float(arrays.get("charge", charge))
    out["mass"] = float(arrays.get("mass", mass))
    return out


# ----------------------------------------------------------------------------
# The slice loop (Sec. 2 enumerate, Fig. 1; Sec. 3.2 predictor-corrector)
# ----------------------------------------------------------------------------

@dataclass
class SweepResult:
    """What a sweep returns (the outputs of the Sec. 2 slice loop)."""
    fields: dict = field(default_factory=dict)      # name -> (n_slices, ny, nx)
    pc_residual: list = field(default_factory=list)  # per slice, last P-C iteration
    removed: int = 0
    plasma: dict = field(default_factory=dict)       # plasma state after the last slice
    beams: list = field(default_factory=list)        # beams after the push (dt != 0)
    witness: dict = field(default_factory=dict)      # beam index -> (sum qw, sum qw Ez, sum qw Ez^2)
    plasma_at: dict = field(default_factory=dict)    # slice -> plasma state at that slice
    plasma_species: list = field(default_factory=list)  # every species' state after the last slice


def _add_fields(a, b):
    return [x + y for x, y in zip(a, b)]


def _sum_species(parts):
    """Componentwise sum of per-species field lists (one species: its list itself, no added zeros)."""
    out = parts[0]
    for p_ in parts[1:]:
        out = _add_fields(out, p_)
    return out


class SliceLoop:
    """The slice loop's state and per-slice body (Sec. 2 enumerate, Fig. 1; Sec. 3.2
    predictor-corrector), one slice per call: the plasma slice of every species with its AB5
    history, the previous slices' plasma J_perp, beam J_perp and B_perp, and the deposit of the
    slice about to be solved.  ``sweep`` drives it over the whole box; the temporal pipeline of
    Sec. 5.2 drives it box by box with the beam handed over from the previous time step.

    Per slice i (``slice``): deposit plasma (all species) + immobile backgrounds + beam(i);
    solve psi -> ExmBy, EypBx; Ez; Bz; predictor-corrector (or the explicit solver) for Bx, By;
    final gather; push the beam particles of slice i; final AB5 step of every plasma species to
    slice i + 1 (each with its own q/M).
    """

    def __init__(self, spec: GridSpec, n0_scale: Optional[torch.Tensor] = None,
                 radial_profile: Optional[torch.Tensor] = None, plasma_perm: Optional[torch.Tensor] = None,
                 reverse_ion_order: bool = False, deposit_noise: float = 0.0, noise_seed: int = 0):
        self.spec = spec
        self.species = plasma_species(spec)
        sts = []
        for k, sp_ in enumerate(self.species):
            st = plasma_init(spec, n0_scale, radial_profile) if not spec.species else plasma_init(spec, species=sp_)
            if plasma_perm is not None and k == 0:
                st = {kk: v[plasma_perm] for kk, v in st.items()}
            sts.append(st)
        bgs = [ion_background(spec, st, q=sp_.charge, reverse=reverse_ion_order)
               for sp_, st in zip(self.species, sts) if sp_.neutralize]
        rho_ion = _sum_species([[b] for b in bgs])[0] if bgs else torch.zeros(spec.ny, spec.nx, dtype=DT)
        self.gen = torch.Generator().manual_seed(noise_seed)
        self.deposit_noise = deposit_noise
        self.rho_ion = self.noisy([rho_ion])[0]
        zero = torch.zeros(spec.ny, spec.nx, dtype=DT)
        self.zero = zero
        # f_{i-1} .. f_{i-4} per species
        self.hists = [[(torch.zeros_like(st["x"]),) * 5 for _ in range(4)] for st in sts]
        self.jx_prev, self.jy_prev = zero, zero
        self.bj_prev = (zero, zero)   # beam J_perp of slice i-1 (explicit solver)
        self.b1 = (zero, zero)
        self.b2 = (zero, zero)
        self.sts = sts
        self.src = self._deposit_full()

    @property
    def st(self):
        """The first species' plasma state (the only one of the default plasma).
        Sec. 3.2 (plasma particle state)."""
        return self.sts[0]

    def _deposit_full(self):
        return self.noisy(_sum_species([plasma_deposit_full(self.spec, st, sp_.charge, sp_.mass)
                                        for sp_, st in zip(self.species, self.sts)]))

    def noisy(self, fields):
        """A test knob: every deposited value times (1 + deposit_noise u), u uniform in [-1, 1]."""
        if self.deposit_noise <= 0.0:
            return fields
        return [f * (1.0 + self.deposit_noise * (2.0 * torch.rand(f.shape, generator=self.gen, dtype=DT) - 1.0))
                for f in fields]

    def slice(self, i: int, cur: Sequence[tuple], nxt: Sequence[tuple], dt: float = 0.0,
              witness: Sequence[int] = ()):
        """Solves slice i.  cur: (beam, sel) pairs, the beam particles `sel` of slice i (one per
        beam); nxt: the same for slice i + 1 (their J_perp enters the predictor-corrector);
        witness: indices into cur whose sums q w (1, Ez, Ez^2) are returned.  Returns (fields,
        last P-C residual, cur's beams after the push of dt (unchanged for dt = 0), witness sums).
        Sec. 2 (the per-slice routine) with Sec. 3.2 (predictor-corrector or explicit B_perp solver)."""
        spec, zero = self.spec, self.zero
        dz = spec.dzeta
        sts, hists, species = self.sts, self.hists, self.species
        rho, jx, jy, jz, chi = self.src
        rho = rho + self.rho_ion
        bj_cur = (zero, zero)
        for b, sel in cur:
            brho, bjx, bjy, bjz = beam_deposit_slice(spec, b, sel)
            rho, jx, jy, jz = rho + brho, jx + bjx, jy + bjy, jz + bjz
            bj_cur = (bj_cur[0] + bjx, bj_cur[1] + bjy)
        psi = poisson_solve(spec, -(rho - jz))
        exmby, eypbx = -ddx(spec, psi), -ddy(spec, psi)
        ez = poisson_solve(spec, ddx(spec, jx) + ddy(spec, jy))
        bz = poisson_solve(spec, ddy(spec, jx) - ddx(spec, jy))
        b1, b2 = self.b1, self.b2
        bx, by = 2.0 * b1[0] - b2[0], 2.0 * b1[1] - b2[1]
        sbx0, sby0 = -ddy(spec, jz), ddx(spec, jz)
        njx, njy = zero, zero
        if i + 1 < spec.nzeta:
            for b, sel in nxt:
                tjx, tjy = beam_deposit_slice(spec, b, sel, ("jx", "jy"))
                njx, njy = njx + tjx, njy + tjy
        resid = 0.0
        if spec.bperp_solver == "explicit":
            # explicit solver: (L - chi) Bx = -dy Jz + Ty, (L - chi) By = dx Jz - Tx with T the
            # B-independent part of d(J_perp)/d(zeta) (explicit_sources; beams by central differences)
            parts = []
            for sp_, st in zip(species, sts):
                F4 = gather(spec, st["x"], st["y"], (exmby, eypbx, ez, bz), spec.shape_order)
                parts.append(explicit_sources(spec, st, F4, sp_.charge, sp_.mass))
            fx, fy, jxx, jxy, jyy = self.noisy(_sum_species(parts))
            tx = fx + ddx(spec, jxx) + ddy(spec, jxy) + (self.bj_prev[0] - njx) / (2.0 * dz)
            ty = fy + ddx(spec, jxy) + ddy(spec, jyy) + (self.bj_prev[1] - njy) / (2.0 * dz)
            (bx, by), rr = helmholtz_pcg(spec, chi, (sbx0 + ty, sby0 - tx), (bx, by), explicit_shift(spec),
                                         spec.n_pc_iter)
            resid = max(rr)
        for _m in range(spec.n_pc_iter if spec.bperp_solver == "pc" else 0):
            parts = []
            for sp_, st, hist in zip(species, sts, hists):
                F = gather(spec, st["x"], st["y"], (exmby, eypbx, ez, bx, by, bz), spec.shape_order)
                f = derivs(sp_.charge / sp_.mass, st["ux"], st["uy"], st["psi"], F)
                tx, ty, tux, tuy, tpsi = ab5_step((st["x"], st["y"], st["ux"], st["uy"], st["psi"]),
                                                  [f] + hist, dz)
                ok = st["alive"] & _state_ok(spec, tx, ty, tpsi)
                parts.append(plasma_deposit_jperp(spec, tx, ty, tux, tuy, tpsi, st["w"], ok, q=sp_.charge))
            pjx, pjy = self.noisy(_sum_species(parts))
            jx1, jy1 = pjx + njx, pjy + njy
            dzjx, dzjy = (self.jx_prev - jx1) / (2.0 * dz), (self.jy_prev - jy1) / (2.0 * dz)
            bxs = poisson_solve(spec, sbx0 + dzjy)
            bys = poisson_solve(spec, sby0 - dzjx)
            nbx = spec.pc_mix * bxs + (1.0 - spec.pc_mix) * bx
            nby = spec.pc_mix * bys + (1.0 - spec.pc_mix) * by
            num = torch.sqrt(((nbx - bx) ** 2).sum() + ((nby - by) ** 2).sum()).detach()
            den = torch.sqrt((nbx ** 2).sum() + (nby ** 2).sum()).detach()
            resid = float(num / den) if float(den) > 0 else 0.0
            bx, by = nbx, nby
        Fs = (exmby, eypbx, ez, bx, by, bz)
        out = dict(rho=rho, jx=jx, jy=jy, jz=jz, chi=chi, psi=psi, exmby=exmby, eypbx=eypbx,
                   ez=ez, bx=bx, by=by, bz=bz)
        wsums = []
        for wi in witness:
            b, sel = cur[wi]
            (ezw,) = gather(spec, b["x"][sel], b["y"][sel], (ez,), spec.shape_order)
            qw = b["charge"] * b["w"][sel]
            wsums.append((qw.sum(), (qw * ezw).sum(), (qw * ezw * ezw).sum()))
        pushed = [beam_push(spec, b, sel, Fs, dt) if dt != 0.0 else b for b, sel in cur]
        # final AB5 step of every species to slice i+1 with the converged fields, removal, deposit
        new_sts, new_hists = [], []
        for sp_, st, hist in zip(species, sts, hists):
            F = gather(spec, st["x"], st["y"], Fs, spec.shape_order)
            f = derivs(sp_.charge / sp_.mass, st["ux"], st["uy"], st["psi"], F)
            nx_, ny_, nux, nuy, npsi = ab5_step((st["x"], st["y"], st["ux"], st["uy"], st["psi"]),
                                                [f] + hist, dz)
            new_hists.append([f] + hist[:3])
            alive = st["alive"] & _state_ok(spec, nx_, ny_, npsi)
            keep = lambda new, old: torch.where(alive, new, old)  # noqa: E731
            new_sts.append(dict(x=keep(nx_, st["x"]), y=keep(ny_, st["y"]), ux=keep(nux, st["ux"]),
                                uy=keep(nuy, st["uy"]), psi=keep(npsi, st["psi"]), w=st["w"], alive=alive))
        self.sts, self.hists = new_sts, new_hists
        self.src = self._deposit_full()
        self.jx_prev, self.jy_prev = jx, jy
        self.bj_prev = bj_cur
        self.b2, self.b1 = b1, (bx, by)
        return out, resid, pushed, wsums


def sweep(spec: GridSpec, beams: Sequence[dict] = (), dt: float = 0.0,
          n_slices: Optional[int] = None, record: Sequence[str] = FIELD_NAMES,
          witness: Sequence[int] = (), record_plasma_at: Sequence[int] = (),
          n0_scale: Optional[torch.Tensor] = None, radial_profile: Optional[torch.Tensor] = None,
          plasma_perm: Optional[torch.Tensor] = None, reverse_ion_order: bool = False,
          deposit_noise: float = 0.0, noise_seed: int = 0,
          crop: Optional[Sequence[int]] = None) -> SweepResult:
    """One quasi-static sweep head -> tail (Sec. 2), slices i = 0 .. n_slices-1 (SliceLoop).

    The beams are binned by slice once, at the start (Sec. 3.1: beam particles sorted per
    slice); dt != 0 advances every beam particle once with its own slice's fields.
    plasma_perm (a permutation of the plasma particles) changes only the order in
    which particle contributions are summed; results are returned in the original order.
    reverse_ion_order sums the ion background in the opposite stencil order, so its
    rounding no longer cancels the electrons' exactly (again the same arithmetic).
    deposit_noise > 0 multiplies every plasma (and ion) deposit node value by
    (1 + deposit_noise * U(-1, 1)): a rounding-size perturbation, like the one an
    unordered (atomic) summation leaves, used to measure the sweep's sensitivity.
    crop = (y0, y1, x0, x1) records only the nodes [y0:y1, x0:x1] of each field (memory).
    """
    ns = spec.nzeta if n_slices is None else n_slices
    loop = SliceLoop(spec, n0_scale, radial_profile, plasma_perm, reverse_ion_order, deposit_noise, noise_seed)
    beams = [dict(b) for b in beams]
    csr = [beam_csr(spec, beam_bins(spec, b["zeta"])) for b in beams]
    sel_of = lambda bi, i: csr[bi][1][csr[bi][0][i]:csr[bi][0][i + 1]]  # noqa: E731

    res = SweepResult()
    rec = {k: [] for k in record}
    wit = {bi: [torch.zeros((), dtype=DT)] * 3 for bi in witness}
    witness = list(witness)
    for i in range(ns):
        if i in record_plasma_at:
            res.plasma_at[i] = {k: v.detach().clone() for k, v in loop.st.items()}
        cur = [(b, sel_of(bi, i)) for bi, b in enumerate(beams)]
        nxt = [(b, sel_of(bi, i + 1)) for bi, b in enumerate(beams)] if i + 1 < spec.nzeta else []
        out, resid, pushed, wsums = loop.slice(i, cur, nxt, dt, witness)
        res.pc_residual.append(resid)
        for k in record:
            rec[k].append(out[k] if crop is None else out[k][crop[0]:crop[1], crop[2]:crop[3]].clone())
        for bi, (w0, w1, w2) in zip(witness, wsums):
            s0, s1, s2 = wit[bi]
            wit[bi] = [s0 + w0, s1 + w1, s2 + w2]
        beams = pushed
    st = loop.st
    res.fields = {k: torch.stack(v) for k, v in rec.items()}
    res.removed = sum(int((~s_["alive"]).sum()) for s_ in loop.sts)
    res.plasma_species = [dict(s_) for s_ in loop.sts]
    if plasma_perm is not None:
        inv = torch.argsort(plasma_perm)
        st = {k: v[inv] for k, v in st.items()}
        res.plasma_species[0] = st
        res.plasma_at = {i: {k: v[inv] for k, v in s_.items()} for i, s_ in res.plasma_at.items()}
    res.plasma = st
    res.beams = beams
    res.witness = {bi: tuple(v) for bi, v in wit.items()}
    return res


def witness_loss(res: SweepResult, beam: int, kind: str = "mean"):
    """Loss of the gradient workloads from the witness sums (S0, S1, S2) = sum(q w (1, Ez, Ez^2)):
    "mean": charge-weighted mean Ez, S1/S0; "mean+rms": that plus the charge-weighted RMS spread
    sqrt(S2/S0 - (S1/S0)^2).  The gradient workloads' losses (a reading: the paper prints no adjoint formulation)."""
    s0, s1, s2 = res.witness[beam]
    mean = s1 / s0
    if kind == "mean":
        return mean
    return mean + torch.sqrt(torch.clamp(s2 / s0 - mean * mean, min=0.0))
