"""Sparse PML Helmholtz operator, sources and receivers (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Discretisation of D = -Z d/dx (1/X) d/dx - X d/dz (1/Z) d/dz - omega^2 gamma X Z
(Sec. 2, eq. helmholtz_preliminary) by the second-order 5-point scheme with the
stretching functions at half nodes.  For node (i, j) (i along x, j along z):

  (A u)_ij = Z_j/h^2 [ (u_ij - u_i+1,j)/X_i+1/2 + (u_ij - u_i-1,j)/X_i-1/2 ]
           + X_i/h^2 [ (u_ij - u_i,j+1)/Z_j+1/2 + (u_ij - u_i,j-1)/Z_j-1/2 ]
           - omega^2 gamma_ij X_i Z_j u_ij ,

with u = 0 on the ghost ring.  The east coefficient of node i equals the west
coefficient of node i+1, so A^T = A (complex symmetric) and A^H v = conj(A conj v).
Without the layer (X = Z = 1) this is -Delta_h - omega^2 diag(gamma) (Sec. 2,
the real symmetric indefinite case).

The solver works with the h^2-scaled operator A' = h^2 A (an exact rescaling
that makes the stencil entries O(1)); the unit point source of amplitude a
then has right-hand side a * e_src (f = a/h^2 at the source node, a discrete
Dirac delta).  ``shift`` beta replaces omega^2 by (1 + i beta) omega^2 (the
shifted operator used by the inner preconditioner).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import grid as G


def level_gamma(grid, gamma_pad: np.ndarray, level: int) -> np.ndarray:
    """gamma on multigrid level ``level``: repeated normalised full weighting,
    coarse node (I, J) <- fine nodes (2I+1+a, 2J+1+b), a, b in {-1, 0, 1}, with
    weights (1,2,1)x(1,2,1)/16 over the nodes that exist."""
    g = np.asarray(gamma_pad, dtype=np.float64)
    w1 = np.array([1.0, 2.0, 1.0])
    for _ in range(level):
        nz, nx = g.shape
        nzc, nxc = nz // 2, nx // 2
        gp = np.pad(g, 1)                        # zero ghost ring
        ones = np.pad(np.ones_like(g), 1)
        acc = np.zeros((nzc, nxc))
        wsum = np.zeros((nzc, nxc))
        J = np.arange(nzc)[:, None]
        I = np.arange(nxc)[None, :]
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                w = w1[a + 1] * w1[b + 1]
                acc += w * gp[2 * J + 1 + b + 1, 2 * I + 1 + a + 1]
                wsum += w * ones[2 * J + 1 + b + 1, 2 * I + 1 + a + 1]
        g = acc / wsum
    return g


def stencil_coefficients(grid, omega: float, gamma_level: np.ndarray, level: int = 0,
                         shift: float = 0.0, sigma_cap: float | None = None):
    """Coefficient arrays (cc, ce, cw, cs, cn), each [Nz_l, Nx_l], of the
    h_l^2-scaled operator of level ``level``: row (j, i) reads
    cc u_ij + ce u_i+1,j + cw u_i-1,j + cs u_i,j+1 + cn u_i,j-1."""
    pa = G.stretch_arrays(grid, omega, level, sigma_cap)
    X, Xh, Z, Zh, nx, nz, h = pa["X"], pa["Xh"], pa["Z"], pa["Zh"], pa["nx"], pa["nz"], pa["h"]
    assert gamma_level.shape == (nz, nx)
    Zc = Z[:, None]
    Xc = X[None, :]
    ce = -Zc / Xh[None, 1:]
    cw = -Zc / Xh[None, :-1]
    cs = -Xc / Zh[1:, None]
    cn = -Xc / Zh[:-1, None]
    ce, cw, cs, cn = (np.broadcast_to(c, (nz, nx)).astype(np.complex128) for c in (ce, cw, cs, cn))
    mass = (1.0 + 1j * shift) * (omega * h) ** 2
    cc = -(ce + cw + cs + cn) - mass * gamma_level * Xc * Zc
    return cc, ce, cw, cs, cn


def assemble(grid, omega: float, gamma_level: np.ndarray, level: int = 0, shift: float = 0.0,
             scaled: bool = True, sigma_cap: float | None = None) -> sp.csr_matrix:
    """The 5-point operator of level ``level`` as a CSR matrix (flat index
    j*Nx_l + i).  ``scaled`` multiplies by h_l^2; neighbours on the ghost ring
    are dropped (u = 0 there)."""
    cc, ce, cw, cs, cn = stencil_coefficients(grid, omega, gamma_level, level, shift, sigma_cap)
    nz, nx = cc.shape
    h = G.stretch_arrays(grid, omega, level)["h"]
    s = 1.0 if scaled else 1.0 / (h * h)
    k = np.arange(nz * nx).reshape(nz, nx)
    rows = [k.ravel()]
    cols = [k.ravel()]
    vals = [cc.ravel()]
    for c, di, dj in ((ce, 1, 0), (cw, -1, 0), (cs, 0, 1), (cn, 0, -1)):
        jj, ii = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        ok = (ii + di >= 0) & (ii + di < nx) & (jj + dj >= 0) & (jj + dj < nz)
        rows.append(k[ok])
        cols.append((k + dj * nx + di)[ok])
        vals.append(c[ok])
    n = nx * nz
    return sp.csr_matrix((np.concatenate(vals) * s, (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def source_vector(grid, ix: int, iz: int, amp: complex) -> np.ndarray:
    """Right-hand side of the h^2-scaled system for a point source of amplitude
    ``amp`` at core node (ix, iz): amp * e_src (f = amp/h^2 times h^2)."""
    Nz, Nx = G.padded_shape(grid)
    f = np.zeros(Nz * Nx, dtype=np.complex128)
    f[G.padded_index(grid, ix, iz)] = amp
    return f


def receiver_indices(grid, survey, k: int) -> np.ndarray:
    """Padded flat indices of the receivers of source k (observation operator Q_k
    of Sec. 2: sampling at receiver nodes)."""
    lo, hi = survey.rec_offsets[k], survey.rec_offsets[k + 1]
    return G.padded_index(grid, survey.rec_ix[lo:hi], survey.rec_iz[lo:hi])


def receiver_weights(survey, k: int) -> np.ndarray:
    lo, hi = survey.rec_offsets[k], survey.rec_offsets[k + 1]
    return np.asarray(survey.rec_w[lo:hi], dtype=np.float64)
