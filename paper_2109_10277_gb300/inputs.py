"""Seeded synthetic workloads shaped like the paper's (arXiv:2109.10277, Sec. 4 and Appendix).

This module holds input recipes only (grid/box parameters and beam particle
draws); none of the method's arithmetic lives here.  Both the CUDA path and the
FP64 oracle are fed from it.

Beams follow the Appendix: Gaussian drivers/witnesses at waist (u_perp = 0),
either random positions with fixed weights (numpy PCG64, seeded) or one particle
per (cell, slice) with a variable weight.  Peak densities are in units of n0.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

GAMMA_DRIVER = 10.0e9 / 0.51099895e6    # 10 GeV electrons (Appendix)
GAMMA_WITNESS = 1.0e9 / 0.51099895e6    # 1 GeV electrons (Appendix)
SEED_DRIVER = 1001
SEED_WITNESS = 1002


def grid_params(name: str) -> dict:
    """Grid/box/solver parameters of a named workload (plain values)."""
    if name == "linear64":      # 64^2 x 64 slices, +-6, FP64, linear shape, 1 ppc
        return dict(nx=64, ny=64, nzeta=64, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0,
                    zeta_min=-7.0, zeta_max=5.0, shape_order=1, ppc_x=1, ppc_y=1,
                    n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    if name == "blowout512":    # 512^2 x 1024 slices, +-8, quadratic, 1 ppc
        return dict(nx=512, ny=512, nzeta=1024, xmin=-8.0, xmax=8.0, ymin=-8.0, ymax=8.0,
                    zeta_min=-13.0, zeta_max=7.0, shape_order=2, ppc_x=1, ppc_y=1,
                    n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    if name == "cubic1024":     # 1024^2 x 1024 slices, +-10, cubic, 4 ppc
        return dict(nx=1024, ny=1024, nzeta=1024, xmin=-10.0, xmax=10.0, ymin=-10.0, ymax=10.0,
                    zeta_min=-18.0, zeta_max=6.0, shape_order=3, ppc_x=2, ppc_y=2,
                    n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    if name == "adjoint256":    # 256^2 x 512 slices, +-6, linear, 1 ppc
        return dict(nx=256, ny=256, nzeta=512, xmin=-6.0, xmax=6.0, ymin=-6.0, ymax=6.0,
                    zeta_min=-7.0, zeta_max=5.0, shape_order=1, ppc_x=1, ppc_y=1,
                    n_pc_iter=5, pc_mix=0.05, psi_guard=0.02)
    if name == "adjoint512":    # 512^2 x 1024 slices, +-8, quadratic, 2 ppc, radial profile
        return dict(nx=512, ny=512, nzeta=1024, xmin=-8.0, xmax=8.0, ymin=-8.0, ymax=8.0,
                    zeta_min=-13.0, zeta_max=7.0, shape_order=2, ppc_x=2, ppc_y=1,
                    n_pc_iter=5, pc_mix=0.05, psi_guard=0.02,
                    radial_profile=[1.0] * 256, profile_rmax=math.sqrt(2.0) * 8.0)
    raise KeyError(name)


def scaled_grid(base: dict, nx: int, ny: int, nzeta: int, **over) -> dict:
    """Same box as `base` with a different resolution (for small parity cases)."""
    g = dict(base)
    g.update(nx=nx, ny=ny, nzeta=nzeta)
    g.update(over)
    return g


def random_beam(n: int, sigma_x: float, sigma_y: float, sigma_z: float, n_peak: float,
                zeta0: float = 0.0, gamma: float = GAMMA_DRIVER, energy_spread: float = 0.0,
                seed: int = SEED_DRIVER, charge: float = -1.0, mass: float = 1.0) -> dict:
    """n fixed-weight particles drawn from a tri-Gaussian (Appendix: random beams).

    Draw order from PCG64(seed): x, y, zeta, energy.  w = n_peak (2 pi)^{3/2} sx sy sz / n.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = sigma_x * rng.standard_normal(n)
    y = sigma_y * rng.standard_normal(n)
    z = zeta0 + sigma_z * rng.standard_normal(n)
    g = gamma * (1.0 + energy_spread * rng.standard_normal(n))
    uz = np.sqrt(np.maximum(g * g - 1.0, 0.0))
    w = np.full(n, n_peak * (2.0 * math.pi) ** 1.5 * sigma_x * sigma_y * sigma_z / n)
    zeros = np.zeros(n)
    return dict(x=x, y=y, zeta=z, ux=zeros.copy(), uy=zeros.copy(), uz=uz, w=w,
                charge=charge, mass=mass)


def fixed_ppc_beam(grid: dict, sigma_r: float, sigma_z: float, n_peak: float, zeta0: float = 0.0,
                   gamma: float = GAMMA_DRIVER, slice_profile: Optional[np.ndarray] = None,
                   extent: float = 5.0, charge: float = -1.0, mass: float = 1.0) -> dict:
    """One particle per (cell, slice) at the cell centre, variable weight (Appendix).

    Cells with |x|, |y| <= extent*sigma_r and |zeta - zeta0| <= extent*sigma_z are
    populated; w = n_b(centre) dx dy dzeta with n_b = n_peak exp(-r^2/2sr^2) exp(-dz^2/2sz^2).
    With `slice_profile` (one entry per slice) the zeta factor n_peak*exp(..) is
    replaced by slice_profile[slice].
    """
    nx, ny, nz = grid["nx"], grid["ny"], grid["nzeta"]
    dx = (grid["xmax"] - grid["xmin"]) / nx
    dy = (grid["ymax"] - grid["ymin"]) / ny
    dz = (grid["zeta_max"] - grid["zeta_min"]) / nz
    xc = grid["xmin"] + (np.arange(nx) + 0.5) * dx
    yc = grid["ymin"] + (np.arange(ny) + 0.5) * dy
    zc = grid["zeta_max"] - (np.arange(nz) + 0.5) * dz
    ix = np.nonzero(np.abs(xc) <= extent * sigma_r)[0]
    iy = np.nonzero(np.abs(yc) <= extent * sigma_r)[0]
    iz = np.nonzero(np.abs(zc - zeta0) <= extent * sigma_z)[0]
    S, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
    S, Y, X = S.reshape(-1), Y.reshape(-1), X.reshape(-1)
    x, y, z = xc[X], yc[Y], zc[S]
    if slice_profile is None:
        zf = n_peak * np.exp(-((z - zeta0) ** 2) / (2.0 * sigma_z ** 2))
    else:
        zf = np.asarray(slice_profile, dtype=np.float64)[S]
    w = zf * np.exp(-(x * x + y * y) / (2.0 * sigma_r ** 2)) * dx * dy * dz
    n = x.size
    zeros = np.zeros(n)
    return dict(x=x, y=y, zeta=z, ux=zeros.copy(), uy=zeros.copy(),
                uz=np.full(n, math.sqrt(gamma * gamma - 1.0)), w=w,
                charge=charge, mass=mass, slice_index=S)


def workload_beams(name: str, n_driver: Optional[int] = None, n_witness: Optional[int] = None,
                   grid: Optional[dict] = None) -> list:
    """Beams of a named workload (seeds 1001 driver, 1002 witness)."""
    grid = grid if grid is not None else grid_params(name)
    if name == "linear64":
        return [random_beam(n_driver or 100_000, 0.3, 0.3, 1.0, 0.01, energy_spread=1e-3)]
    if name == "blowout512":
        return [random_beam(n_driver or 1_000_000, 0.2, 0.2, 1.4, 5.0, energy_spread=1e-3)]
    if name == "cubic1024":
        return [random_beam(n_driver or 10_000_000, 0.15, 0.15, 1.2, 10.0, energy_spread=1e-3),
                random_beam(n_witness or 2_000_000, 0.05, 0.05, 0.3, 20.0, zeta0=-6.0,
                            gamma=GAMMA_WITNESS, seed=SEED_WITNESS)]
    if name == "adjoint256":
        return [fixed_ppc_beam(grid, 0.2, 1.0, 2.0),
                fixed_ppc_beam(grid, 0.1, 0.3, 20.0, zeta0=-5.0, gamma=GAMMA_WITNESS)]
    if name == "adjoint512":
        nz = grid["nzeta"]
        dz = (grid["zeta_max"] - grid["zeta_min"]) / nz
        zc = grid["zeta_max"] - (np.arange(nz) + 0.5) * dz
        prof = 4.0 * np.exp(-zc ** 2 / (2.0 * 1.4 ** 2))
        return [fixed_ppc_beam(grid, 0.2, 1.4, 4.0, slice_profile=prof),
                fixed_ppc_beam(grid, 0.1, 0.3, 20.0, zeta0=-5.0, gamma=GAMMA_WITNESS)]
    raise KeyError(name)
