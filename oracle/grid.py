"""Padded grid, PML stretching functions and model embedding (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2, eq. helmholtz_preliminary: the domain is the core plus a damping layer
where the complex stretching functions X(x), Z(z) differ from 1; U = 0 on the
outer boundary.  The paper does not give the layer profile (it cites Yavich
2021).  Reading used here: ``npml`` nodes on each of the four sides, quadratic
profile sigma(d) = sigma_max (d/L)^2 with L = npml*h and
sigma_max = 3 c ln(1/R) / (2L) (Collino & Tsogka 2001), time convention
e^{-i omega t} so X = 1 + i sigma_x / omega.  The Dirichlet value sits on a
ghost ring one node outside the padded grid.

Multigrid levels (of the inner solver chosen here; the paper has none) reuse the same
continuous profile: level l has spacing h_l = 2^l h, first node at
x0_l = (2^l - 1) h and n_l = floor(n_{l-1} / 2) nodes per direction, so coarse
node I sits on fine node 2I+1 and the ghost nodes of every level coincide with
(or lie one fine node beyond) the fine ghosts.
"""
from __future__ import annotations

import numpy as np


def padded_shape(grid):
    """(Nz, Nx) of the padded grid: core + npml nodes on every side."""
    return grid.nz + 2 * grid.npml, grid.nx + 2 * grid.npml


def sigma_max(grid) -> float:
    """Peak damping of the quadratic profile (Collino & Tsogka 2001)."""
    if grid.npml == 0:
        return 0.0
    L = grid.npml * grid.h
    return 3.0 * grid.pml_c * np.log(1.0 / grid.pml_R) / (2.0 * L)


def sigma_at(grid, pos: np.ndarray, n_core: int) -> np.ndarray:
    """sigma at physical positions ``pos`` (metres from padded node 0) along an
    axis whose core spans padded nodes [npml, npml + n_core - 1]."""
    if grid.npml == 0:
        return np.zeros_like(np.asarray(pos, dtype=np.float64))
    p, h = grid.npml, grid.h
    lo = p * h
    hi = (p + n_core - 1) * h
    d = np.maximum(np.maximum(lo - pos, pos - hi), 0.0)
    L = p * h
    return sigma_max(grid) * (d / L) ** 2


def level_axis(grid, n0: int, level: int):
    """(n_l, x0_l, h_l) of multigrid level ``level`` for an axis with ``n0``
    fine (padded) nodes."""
    n, x0, h = n0, 0.0, grid.h
    for _ in range(level):
        x0 = x0 + h
        h = 2.0 * h
        n = n // 2
    return n, x0, h


def stretch_arrays(grid, omega: float, level: int = 0, sigma_cap: float | None = None):
    """Stretching functions of one level.

    ``sigma_cap`` (used only by the multigrid preconditioner's shifted operator)
    clips sigma/omega at that value.

    Returns dict with complex128 arrays
      X  [Nx_l]      X at nodes,       Xh [Nx_l + 1]  X at half nodes i - 1/2 (i = 0..Nx_l)
      Z  [Nz_l]      Z at nodes,       Zh [Nz_l + 1]  Z at half nodes j - 1/2
    and the level sizes/spacing.  Xh[i] is X_{i-1/2}, so X_{i+1/2} = Xh[i+1].
    """
    Nz0, Nx0 = padded_shape(grid)
    nx_l, x0, h_l = level_axis(grid, Nx0, level)
    nz_l, z0, _ = level_axis(grid, Nz0, level)
    xn = x0 + h_l * np.arange(nx_l)
    xh = x0 + h_l * (np.arange(nx_l + 1) - 0.5)
    zn = z0 + h_l * np.arange(nz_l)
    zh = z0 + h_l * (np.arange(nz_l + 1) - 0.5)
    def stretch(pos, n_core):
        r = sigma_at(grid, pos, n_core) / omega
        if sigma_cap is not None:
            r = np.minimum(r, sigma_cap)
        return 1.0 + 1j * r

    X = stretch(xn, grid.nx)
    Xh = stretch(xh, grid.nx)
    Z = stretch(zn, grid.nz)
    Zh = stretch(zh, grid.nz)
    return dict(X=X, Xh=Xh, Z=Z, Zh=Zh, nx=nx_l, nz=nz_l, h=h_l)


def pad_gamma(grid, gamma_core: np.ndarray) -> np.ndarray:
    """Embed the core model into the padded grid, replicating edge values into
    the damping layer (the layer's gamma is then held fixed; only core values are
    control variables, cf. the sizes of Fig. M)."""
    p = grid.npml
    return np.pad(np.asarray(gamma_core, dtype=np.float64), p, mode="edge")


def core_index(grid) -> np.ndarray:
    """Flat padded indices of the core nodes, core order (z slow, x fast).
    This is the embedding E of the control into the padded grid."""
    Nz, Nx = padded_shape(grid)
    p = grid.npml
    iz, ix = np.meshgrid(np.arange(grid.nz) + p, np.arange(grid.nx) + p, indexing="ij")
    return (iz * Nx + ix).ravel()


def padded_index(grid, ix_core, iz_core) -> np.ndarray:
    """Flat padded index of core node (ix, iz)."""
    Nz, Nx = padded_shape(grid)
    p = grid.npml
    return (np.asarray(iz_core) + p) * Nx + (np.asarray(ix_core) + p)
