"""Pins of the oracle's ILU(0) (the paper's incomplete-LU block approximation
of Sec. 5 with zero fill) against its definition and library routines.
CPU only."""
import numpy as np
import scipy.sparse.linalg as spla

import fwi_inputs as FI
from oracle import fwi
from oracle import grid as G
from oracle.ilu import ILU0


def _op(nx=17, nz=11, npml=4, f=5.0):
    wl = FI.micro_workload(nx=nx, nz=nz, npml=npml, freq=f)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    A = prob.operator(wl.gamma_start.ravel(), 0)
    Nz, Nx = G.padded_shape(wl.grid)
    return A, Nz, Nx


def test_factors_reproduce_the_matrix_on_its_pattern():
    """The defining property of ILU(0): L unit lower and U upper triangular on
    A's pattern, and (L U)_pq = A_pq wherever A_pq != 0; the dropped fill
    lies only on the two diagonals k -/+ (Nx - 1)."""
    A, Nz, Nx = _op()
    F = ILU0(A, Nz, Nx)
    L, U = F.L(), F.U()
    assert abs(L - L.multiply(np.tri(*L.shape, dtype=bool))).max() == 0
    assert np.all(L.diagonal() == 1.0)
    assert abs(U - U.multiply(np.tri(*U.shape, dtype=bool).T)).max() == 0
    LU = (L @ U).tocoo()
    Ad = A.toarray()
    LUd = LU.toarray()
    mask = Ad != 0
    np.testing.assert_allclose(LUd[mask], Ad[mask], rtol=1e-13, atol=1e-13 * np.abs(Ad).max())
    r, c = np.nonzero(np.abs(LUd - Ad) > 1e-12 * np.abs(Ad).max())
    assert set(np.unique(c - r)) <= {Nx - 1, -(Nx - 1)}


def test_solve_equals_triangular_solves_of_the_factors():
    """(L U)^{-1} b by the oracle's substitutions equals scipy's sparse
    triangular solves with the same factors; the adjoint is conj(solve(conj))."""
    A, Nz, Nx = _op()
    F = ILU0(A, Nz, Nx)
    b = np.random.default_rng(0).standard_normal(Nz * Nx) + 1j * np.random.default_rng(1).standard_normal(Nz * Nx)
    y = spla.spsolve_triangular(F.L().tocsr(), b, lower=True)
    x = spla.spsolve_triangular(F.U().tocsr(), y, lower=False)
    np.testing.assert_allclose(F.solve(b), x, rtol=1e-12)
    Lh, Uh = F.L().conj().T.tocsr(), F.U().conj().T.tocsr()
    xa = spla.spsolve_triangular(Lh, spla.spsolve_triangular(Uh, b, lower=True), lower=False)
    np.testing.assert_allclose(F.solve_adjoint(b), xa, rtol=1e-12)


def test_tridiagonal_case_is_exact():
    """With one grid row (Nz = 1) A is tridiagonal, ILU(0) drops nothing and is
    the exact LU: its solve equals a direct sparse solve."""
    A, Nz, Nx = _op(nx=25, nz=3, npml=0)
    # one row of the operator: the tridiagonal block of the first grid row
    A1 = A[:Nx, :Nx]
    F = ILU0(A1, 1, Nx)
    b = np.random.default_rng(2).standard_normal(Nx) + 0j
    np.testing.assert_allclose(F.solve(b), spla.spsolve(A1.tocsc(), b), rtol=1e-12)
