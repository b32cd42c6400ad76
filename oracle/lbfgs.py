"""Limited-memory BFGS approximation of the reduced Hessian in the H block of
the preconditioner (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 5 (after eq. precond) notes that the block-triangular preconditioner
approximates the reduced Hessian H by the regulariser L, and that other
approximations of H, in particular L-BFGS (Biros & Ghattas 2005), can take its
place; Sec. 7 repeats this and names the background Hessian as well.  With the
H block replaced by an approximation B of H, the middle step of the
preconditioner becomes

    z_s = B^{-1} (v2 + Re(P~^H z_lambda))          (instead of ( ... ) / eps).

This module builds B^{-1} by the standard L-BFGS inverse update from stored
pairs (s_i, y_i) with y_i = H s_i (or a secant difference), oldest first, and
the initial inverse H_0 = (1/eps) I, so that with no pairs it is the paper's
L^{-1}.  The product B^{-1} q is the two-loop recursion (Nocedal & Wright,
Numerical Optimization, 2nd ed., Sec. 7.2, Algorithm 7.4): a backward pass
q <- q - alpha_i y_i with alpha_i = rho_i s_i^T q, rho_i = 1 / (y_i^T s_i),
from the newest pair to the oldest; r = H_0 q; a forward pass
r <- r + (alpha_i - rho_i y_i^T r) s_i from the oldest pair to the newest.

``dense_inverse`` is the same matrix built by the textbook update formula
H_{k+1} = V_k^T H_k V_k + rho_k s_k s_k^T, V_k = I - rho_k y_k s_k^T (for
tests on small sizes).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np


def check_pairs(pairs: Sequence[Tuple[np.ndarray, np.ndarray]]):
    """Every pair needs positive curvature s^T y > 0 (B stays positive definite)."""
    for k, (s, y) in enumerate(pairs):
        if not float(np.dot(s, y)) > 0.0:
            raise ValueError(f"pair {k}: s^T y = {float(np.dot(s, y))} is not positive")


def two_loop(q: np.ndarray, pairs: Sequence[Tuple[np.ndarray, np.ndarray]], h0: float) -> np.ndarray:
    """B^{-1} q by the two-loop recursion (pairs oldest first, H_0 = h0 I)."""
    check_pairs(pairs)
    q = np.array(q, dtype=np.float64, copy=True)
    alphas = []
    for s, y in reversed(pairs):               # newest to oldest
        rho = 1.0 / float(np.dot(y, s))
        a = rho * float(np.dot(s, q))
        q -= a * y
        alphas.append(a)
    r = h0 * q
    for (s, y), a in zip(pairs, reversed(alphas)):   # oldest to newest
        rho = 1.0 / float(np.dot(y, s))
        b = rho * float(np.dot(y, r))
        r += (a - b) * s
    return r


def dense_inverse(pairs: Sequence[Tuple[np.ndarray, np.ndarray]], h0: float, n: int) -> np.ndarray:
    """The inverse approximation as a dense n x n matrix, by the BFGS update
    formula applied to the pairs in order (small n only)."""
    check_pairs(pairs)
    Hk = h0 * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / float(np.dot(y, s))
        V = np.eye(n) - rho * np.outer(y, s)
        Hk = V.T @ Hk @ V + rho * np.outer(s, s)
    return Hk
