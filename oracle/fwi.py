"""Forward modelling, data residual, misfit and adjoint gradient (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 (eqs. helmholtz_j, Au=f): one independent Helmholtz problem per source
and frequency; the block index is b = f * n_src + k (frequency major).  Each
frequency's operator is factorised once with scipy's sparse LU, as the paper's
own code does (Sec. 6).  Sec. 3: r = d - Q S(s_n), Phi = 1/2 sum |W r|^2, and
the gradient of Phi with respect to the core squared slowness is
-sum_b omega_b^2 Re(conj(u_b) lambda_b) with A^H lambda_b = Q^T W^T W r_b
(the adjoint-state form of W^T J^* r, eqs. jacobian and G, S, P).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List

import numpy as np
import scipy.sparse.linalg as spla

from . import grid as G
from . import helmholtz as H


@dataclass
class Problem:
    """One instance: grid, survey, the fixed damping-layer model and gamma_ref.

    ``gamma_pad_fixed`` holds the model on the padded grid; its layer values are
    frozen at construction (edge replication of the initial core model) and only
    the core is ever replaced by the control s."""

    grid: object
    survey: object
    gamma_pad_fixed: np.ndarray
    gamma_ref: float
    _lu: Dict = field(default_factory=dict)

    @staticmethod
    def create(grid, survey, gamma_core0: np.ndarray, gamma_ref: float | None = None):
        gp = G.pad_gamma(grid, gamma_core0)
        gref = float(np.mean(gamma_core0)) if gamma_ref is None else float(gamma_ref)
        return Problem(grid, survey, gp, gref)

    @property
    def omegas(self) -> List[float]:
        return [2.0 * np.pi * f for f in self.survey.freqs_hz]

    @property
    def n_blocks(self) -> int:
        return self.survey.n_freq * self.survey.n_src

    def block_freq(self, b: int) -> int:
        return b // self.survey.n_src

    def block_src(self, b: int) -> int:
        return b % self.survey.n_src

    def gamma_pad(self, s_core: np.ndarray) -> np.ndarray:
        g = self.gamma_pad_fixed.copy()
        p = self.grid.npml
        g[p:p + self.grid.nz, p:p + self.grid.nx] = np.asarray(s_core).reshape(self.grid.nz, self.grid.nx)
        return g

    def operator(self, s_core: np.ndarray, f: int, shift: float = 0.0):
        return H.assemble(self.grid, self.omegas[f], self.gamma_pad(s_core), 0, shift)

    def lu(self, s_core: np.ndarray, f: int):
        """Sparse LU of the scaled operator A'_f (cached per model and frequency)."""
        key = (f, hash(np.asarray(s_core, dtype=np.float64).tobytes()))
        if key not in self._lu:
            self._lu = {k: v for k, v in self._lu.items() if k[1] == key[1]}
            self._lu[key] = spla.splu(self.operator(s_core, f).tocsc())
        return self._lu[key]


def solve(prob: Problem, s_core, f: int, rhs: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """A'_f^{-1} rhs, or A'_f^{-H} rhs = conj(A'^{-1} conj(rhs)) (A' symmetric)."""
    lu = prob.lu(s_core, f)
    if adjoint:
        return np.conj(lu.solve(np.conj(rhs)))
    return lu.solve(rhs)


def forward(prob: Problem, s_core) -> np.ndarray:
    """Wavefields u [B, N] (complex128, padded grid flattened z-major)."""
    sv = prob.survey
    out = []
    for f in range(sv.n_freq):
        for k in range(sv.n_src):
            rhs = H.source_vector(prob.grid, int(sv.src_ix[k]), int(sv.src_iz[k]), complex(sv.src_amp[k]))
            out.append(solve(prob, s_core, f, rhs))
    return np.array(out)


def sample(prob: Problem, u: np.ndarray) -> List[np.ndarray]:
    """Q u per block: the wavefield at the block's receivers."""
    return [u[b][H.receiver_indices(prob.grid, prob.survey, prob.block_src(b))]
            for b in range(prob.n_blocks)]


def residual(prob: Problem, u: np.ndarray, d_obs: List[np.ndarray]) -> List[np.ndarray]:
    """r_b = d_b - Q_b u_b."""
    return [d_obs[b] - q for b, q in enumerate(sample(prob, u))]


def misfit(prob: Problem, r: List[np.ndarray]) -> float:
    """Phi = 1/2 sum_b ||W_b r_b||^2."""
    tot = 0.0
    for b, rb in enumerate(r):
        w = H.receiver_weights(prob.survey, prob.block_src(b))
        tot += 0.5 * float(np.sum((w * np.abs(rb)) ** 2))
    return tot


def scatter_weighted(prob: Problem, r: List[np.ndarray]) -> np.ndarray:
    """Q^T W^T W r per block, as padded-grid vectors [B, N]."""
    Nz, Nx = G.padded_shape(prob.grid)
    out = np.zeros((prob.n_blocks, Nz * Nx), dtype=np.complex128)
    for b, rb in enumerate(r):
        k = prob.block_src(b)
        idx = H.receiver_indices(prob.grid, prob.survey, k)
        w = H.receiver_weights(prob.survey, k)
        np.add.at(out[b], idx, w * w * rb)
    return out


def adjoint_fields(prob: Problem, s_core, g: np.ndarray) -> np.ndarray:
    """lambda'_b = A'^{-H} g_b for every block."""
    return np.array([solve(prob, s_core, prob.block_freq(b), g[b], adjoint=True)
                     for b in range(prob.n_blocks)])


def gradient(prob: Problem, s_core, d_obs):
    """(Phi, dPhi/dgamma_core [nz*nx]) at model ``s_core`` (unscaled units).

    With A' = h^2 A the adjoint field of the unscaled system is lambda = h^2 lambda',
    so dPhi/ds_c = -sum_b omega_b^2 h^2 Re(conj(u_b,c) lambda'_b,c)."""
    u = forward(prob, s_core)
    r = residual(prob, u, d_obs)
    phi = misfit(prob, r)
    lam = adjoint_fields(prob, s_core, scatter_weighted(prob, r))
    ci = G.core_index(prob.grid)
    h2 = prob.grid.h ** 2
    g = np.zeros(ci.size)
    for b in range(prob.n_blocks):
        w2 = prob.omegas[prob.block_freq(b)] ** 2
        g -= w2 * h2 * np.real(np.conj(u[b][ci]) * lam[b][ci])
    return phi, g
