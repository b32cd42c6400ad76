"""Geometric multigrid for the shifted PML Helmholtz operator (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper approximates A inside eq. precond_approx by an incomplete LU and
names a shifted-Laplacian preconditioner with multigrid (Erlangga et al.) as
the better choice (Sec. 5); it gives no multigrid details.  The design below
is this package's own choice, stated as plainly as possible so that the CUDA kernels can
be compared with it element by element; the tests pin it against the exact
Fourier symbols of the cycle on constant-coefficient grids without the layer:

  * operator of level l: the h_l^2-scaled 5-point PML operator rediscretised
    on level l with omega^2 -> (1 + i beta) omega^2 (helmholtz.assemble with
    ``shift``), gamma by normalised full weighting (helmholtz.level_gamma);
  * coarse node I on fine node 2I+1; prolongation P bilinear (weights 1 on the
    coinciding node, 1/2 on edge neighbours, 1/4 on diagonal ones, zero
    ghosts); restriction R = P^T, which is 4x full weighting, the factor 4
    being h_{l+1}^2 / h_l^2 of the scaled operators;
  * the shifted operator clips the layer's sigma/omega at ``sigma_cap``
    (default 1): with sigma/omega > 1 the stretched rows stop being
    diagonally dominant and damped Jacobi amplifies modes that are smooth
    along the layer and rough across it, which no coarse grid removes;
  * smoother: damped Jacobi, x <- x + w D^{-1} (b - M x);
  * coarsest level: exact dense solve;
  * cycle index ``cycle`` (1 = V, 2 = W) on levels 1..``wdepth`` and V below
    (the coarse levels, where the shifted operator is nearly diagonal, gain
    nothing from repeated corrections), (nu1, nu2) sweeps, zero initial guess.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import grid as G
from . import helmholtz as H


def prolong_1d(n_f: int, n_c: int) -> sp.csr_matrix:
    """1D linear interpolation from n_c coarse nodes (coarse I at fine 2I+1)."""
    rows, cols, vals = [], [], []
    for I in range(n_c):
        for i, w in ((2 * I, 0.5), (2 * I + 1, 1.0), (2 * I + 2, 0.5)):
            if 0 <= i < n_f:
                rows.append(i); cols.append(I); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, n_c))


def level_shapes(grid, levels: int):
    Nz, Nx = G.padded_shape(grid)
    out = []
    for l in range(levels):
        out.append((G.level_axis(grid, Nz, l)[0], G.level_axis(grid, Nx, l)[0]))
    return out


def auto_levels(grid, max_coarse_nodes: int = 256, min_dim: int = 3) -> int:
    """Number of levels (fine included): coarsen while the current level has more
    than ``max_coarse_nodes`` nodes and the next level keeps >= ``min_dim`` nodes
    in both directions."""
    Nz, Nx = G.padded_shape(grid)
    levels = 1
    nz, nx = Nz, Nx
    while nz * nx > max_coarse_nodes and nz // 2 >= min_dim and nx // 2 >= min_dim:
        nz, nx = nz // 2, nx // 2
        levels += 1
    return levels


class Hierarchy:
    """Operators, transfers and the coarsest inverse for one (omega, gamma)."""

    def __init__(self, grid, omega: float, gamma_pad: np.ndarray, shift: float = 0.5,
                 levels: int | None = None, nu1: int = 2, nu2: int = 2, wj: float = 0.5,
                 cycle: int = 2, sigma_cap: float | None = 1.0, wdepth: int = 2):
        self.grid = grid
        self.levels = auto_levels(grid) if levels is None else int(levels)
        self.shapes = level_shapes(grid, self.levels)
        self.nu1, self.nu2, self.wj, self.cycle, self.wdepth = nu1, nu2, wj, cycle, wdepth
        self.gammas = [H.level_gamma(grid, gamma_pad, l) for l in range(self.levels)]
        self.ops = [H.assemble(grid, omega, self.gammas[l], l, shift, sigma_cap=sigma_cap)
                    for l in range(self.levels)]
        self.diag = [op.diagonal() for op in self.ops]
        self.P = []
        for l in range(self.levels - 1):
            (nzf, nxf), (nzc, nxc) = self.shapes[l], self.shapes[l + 1]
            self.P.append(sp.kron(prolong_1d(nzf, nzc), prolong_1d(nxf, nxc)).tocsr())
        self.coarse_inv = np.linalg.inv(self.ops[-1].toarray())

    def smooth(self, l: int, x: np.ndarray, b: np.ndarray, sweeps: int) -> np.ndarray:
        for _ in range(sweeps):
            x = x + self.wj * (b - self.ops[l] @ x) / self.diag[l]
        return x

    def restrict(self, l: int, r: np.ndarray) -> np.ndarray:
        return self.P[l].T @ r

    def prolong(self, l: int, e: np.ndarray) -> np.ndarray:
        return self.P[l] @ e

    def vcycle(self, b: np.ndarray, l: int = 0) -> np.ndarray:
        """One multigrid cycle with (nu1, nu2) Jacobi sweeps for M_l x = b from
        x = 0.  The fine level (l = 0) does one coarse-grid correction; levels
        1..wdepth repeat theirs ``cycle`` times (W for cycle = 2); deeper
        levels do one (V)."""
        if l == self.levels - 1:
            return self.coarse_inv @ b
        x = self.smooth(l, np.zeros_like(b), b, self.nu1)
        for _ in range(self.cycle if 0 < l <= self.wdepth else 1):
            rc = self.restrict(l, b - self.ops[l] @ x)
            x = x + self.prolong(l, self.vcycle(rc, l + 1))
        return self.smooth(l, x, b, self.nu2)


def inner_solve(A, hier: Hierarchy, rhs: np.ndarray, iters: int, adjoint: bool = False,
                tol: float = 0.0):
    """The inexact block solve of the preconditioner: right-preconditioned
    BiCGStab on A' with one V-cycle of the shifted operator as preconditioner.
    The adjoint solve uses A'^H = conj(A') and conj(V-cycle(conj .)), i.e. it is
    conj(solve(conj(rhs)))."""
    from .krylov import bicgstab
    if adjoint:
        x, hist = inner_solve(A, hier, np.conj(rhs), iters, False, tol)
        return np.conj(x), hist
    return bicgstab(lambda v: A @ v, rhs, hier.vcycle, iters=iters, tol=tol)
