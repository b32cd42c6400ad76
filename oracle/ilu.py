"""Incomplete LU factorisation with zero fill, ILU(0), of the 5-point operator
(oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 5 (after eq. precond_approx) approximates the Helmholtz blocks A by an
incomplete LU factorisation (Sec. 6 uses a fill-in level of 21 in the paper's
CPU code).  This module restates the zero-fill variant for the 5-point
operator in the natural ordering (flat index k = j*Nx + i): L unit lower
triangular and U upper triangular, both with the sparsity pattern of A, such
that (L U)_pq = A_pq for every (p, q) in the pattern of A (the definition of
ILU(0)).  With the row-major ordering the only couplings below the diagonal
are west (k-1) and north (k-Nx), so

    U_{k,k+1} = A_{k,k+1},  U_{k,k+Nx} = A_{k,k+Nx},
    L_{k,k-1} = A_{k,k-1} / d_{k-1},  L_{k,k-Nx} = A_{k,k-Nx} / d_{k-Nx},
    d_k = A_kk - L_{k,k-1} U_{k-1,k} - L_{k,k-Nx} U_{k-Nx,k},

(the products that would land on k-Nx+1 and k+Nx-1 are the dropped fill).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class ILU0:
    """ILU(0) factors of a 5-point operator on an Nz x Nx grid (CSR input)."""

    def __init__(self, A: sp.csr_matrix, nz: int, nx: int):
        A = sp.csr_matrix(A)
        n = nz * nx
        self.nz, self.nx, self.n = nz, nx, n
        diag = A.diagonal().astype(np.complex128)

        def coef(di, dj):
            """A[k, k + dj*nx + di] for every k (0 where the neighbour is outside)."""
            out = np.zeros(n, dtype=np.complex128)
            k = np.arange(n)
            j, i = np.divmod(k, nx)
            ok = (i + di >= 0) & (i + di < nx) & (j + dj >= 0) & (j + dj < nz)
            out[ok] = np.asarray(A[k[ok], (k + dj * nx + di)[ok]]).ravel()
            return out
        self.ce, self.cw, self.cs, self.cn = coef(1, 0), coef(-1, 0), coef(0, 1), coef(0, -1)
        d = np.zeros(n, dtype=np.complex128)
        lw = np.zeros(n, dtype=np.complex128)
        ln = np.zeros(n, dtype=np.complex128)
        for k in range(n):                       # the recurrence in the natural order
            dk = diag[k]
            if k % nx > 0:
                lw[k] = self.cw[k] / d[k - 1]
                dk = dk - lw[k] * self.ce[k - 1]
            if k >= nx:
                ln[k] = self.cn[k] / d[k - nx]
                dk = dk - ln[k] * self.cs[k - nx]
            d[k] = dk
        self.d, self.lw, self.ln = d, lw, ln

    def L(self) -> sp.csr_matrix:
        n, nx = self.n, self.nx
        k = np.arange(n)
        rows = np.concatenate([k, k[k % nx > 0], k[k >= nx]])
        cols = np.concatenate([k, k[k % nx > 0] - 1, k[k >= nx] - nx])
        vals = np.concatenate([np.ones(n), self.lw[k % nx > 0], self.ln[k >= nx]])
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    def U(self) -> sp.csr_matrix:
        n, nx = self.n, self.nx
        k = np.arange(n)
        e = k % nx < nx - 1
        s = k < n - nx
        rows = np.concatenate([k, k[e], k[s]])
        cols = np.concatenate([k, k[e] + 1, k[s] + nx])
        vals = np.concatenate([self.d, self.ce[e], self.cs[s]])
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    def solve(self, b: np.ndarray) -> np.ndarray:
        """(L U)^{-1} b: forward substitution with L, backward with U, in the
        natural order."""
        n, nx = self.n, self.nx
        y = np.array(b, dtype=np.complex128)
        for k in range(n):
            if k % nx > 0:
                y[k] -= self.lw[k] * y[k - 1]
            if k >= nx:
                y[k] -= self.ln[k] * y[k - nx]
        x = np.zeros(n, dtype=np.complex128)
        for k in range(n - 1, -1, -1):
            acc = y[k]
            if k % nx < nx - 1:
                acc -= self.ce[k] * x[k + 1]
            if k + nx < n:
                acc -= self.cs[k] * x[k + nx]
            x[k] = acc / self.d[k]
        return x

    def solve_adjoint(self, b: np.ndarray) -> np.ndarray:
        """(L U)^{-H} applied as conj((L U)^{-1} conj b): A is complex symmetric
        and the factors of conj(A) are the conjugated factors, so this is the
        ILU(0) approximation of A^{-H} that the adjoint block solves use."""
        return np.conj(self.solve(np.conj(b)))
