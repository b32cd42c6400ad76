"""The KKT system of one Gauss-Newton step and its preconditioners (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4, eq. KKT: with F = Q^T W^T W Q, L = eps I and P = omega^2 diag(u_n),

    [ F   0    A^* ] [du]   [ Q^T W^T W r ]
    [ 0   L   -P^* ] [ds] = [ -L s_n      ]
    [ A  -P    0   ] [lm]   [ 0           ]

Readings (the paper leaves these open):
  * the control ds is real (gamma is real, Sec. 2); row 2 is then
    eps ds - Re(P^* lambda) and the system is real-linear and symmetric in the
    real inner product <x, y> = Re(x^H y) (a plain dot over interleaved re/im);
  * the control lives on the core nodes only (the L block of Fig. M is smaller
    than the A blocks): P_b = omega_b^2 diag(u_b) E with E the core embedding;
  * exact rescaling used by both this oracle and the CUDA path: A' = h^2 A,
    lambda' = lambda / h^2, control ds~ = ds / gamma_ref, so
    P~_b = h^2 gamma_ref omega_b^2 diag(u_b) E; the regulariser is measured on
    the relative model, (eps/2) ||(s_n + ds)/gamma_ref||^2, i.e. the paper's
    eps equals this eps / gamma_ref^2.  The scaled system reads

    [ F    0    A'^H ] [du ]   [ Q^T W^2 r        ]
    [ 0   eps  -P~^H ] [ds~] = [ -eps s_n/gamma_ref ]   (row 2 real part only)
    [ A'  -P~    0   ] [lm']   [ 0                ]

Preconditioner (Sec. 5, eq. precond): P = [[0,0,A^*],[0,L,-P^*],[A,-P,0]] is
block triangular after permutation, so P z = v is solved by
z_lm = A'^{-H} v1, z_s = (v2 + Re(P~^H z_lm)) / eps, z_u = A'^{-1}(v3 + P~ z_s).
eq. precond_approx replaces A' by an approximation (``inner``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fwi
from . import grid as G
from . import helmholtz as H


class KKT:
    """The scaled KKT system of one instance at the model ``s_n``."""

    def __init__(self, prob: fwi.Problem, s_n: np.ndarray, d_obs, eps: float,
                 include_Ls_n: bool = True, u_n: np.ndarray | None = None):
        self.prob = prob
        self.s_n = np.asarray(s_n, dtype=np.float64).ravel()
        self.eps = float(eps)
        self.include_Ls_n = bool(include_Ls_n)
        self.u = fwi.forward(prob, self.s_n) if u_n is None else u_n
        self.r = fwi.residual(prob, self.u, d_obs)
        self.B = prob.n_blocks
        Nz, Nx = G.padded_shape(prob.grid)
        self.N = Nz * Nx
        self.ci = G.core_index(prob.grid)
        self.Nc = self.ci.size
        h2 = prob.grid.h ** 2
        self.c = np.array([h2 * prob.gamma_ref * prob.omegas[prob.block_freq(b)] ** 2 * self.u[b]
                           for b in range(self.B)])           # P~_b = diag(c_b) E
        self.Fd = np.zeros((self.B, self.N))                   # diagonal of F_b
        for b in range(self.B):
            k = prob.block_src(b)
            np.add.at(self.Fd[b], H.receiver_indices(prob.grid, prob.survey, k),
                      H.receiver_weights(prob.survey, k) ** 2)
        self.A = [prob.operator(self.s_n, f) for f in range(prob.survey.n_freq)]

    # ---------------------------------------------------------------- layout
    def pack(self, du, ds, lm) -> np.ndarray:
        """Flat real vector [du (re,im interleaved, block major), lm (same), ds]."""
        return np.concatenate([np.ascontiguousarray(du, dtype=np.complex128).view(np.float64).ravel(),
                               np.ascontiguousarray(lm, dtype=np.complex128).view(np.float64).ravel(),
                               np.asarray(ds, dtype=np.float64).ravel()])

    def unpack(self, x: np.ndarray):
        n = 2 * self.B * self.N
        du = x[:n].view(np.complex128).reshape(self.B, self.N)
        lm = x[n:2 * n].view(np.complex128).reshape(self.B, self.N)
        ds = x[2 * n:]
        return du, ds, lm

    @property
    def size(self) -> int:
        return 4 * self.B * self.N + self.Nc

    # ---------------------------------------------------------------- blocks
    def Aop(self, b, x, adjoint=False):
        A = self.A[self.prob.block_freq(b)]
        return np.conj(A @ np.conj(x)) if adjoint else A @ x

    def P_apply(self, b, ds):
        """P~_b ds (complex, padded grid)."""
        out = np.zeros(self.N, dtype=np.complex128)
        out[self.ci] = self.c[b][self.ci] * ds
        return out

    def PH_apply_re(self, b, lm_b):
        """Re(P~_b^H lm_b) on the core."""
        return np.real(np.conj(self.c[b][self.ci]) * lm_b[self.ci])

    # ---------------------------------------------------------------- system
    def matvec(self, x: np.ndarray) -> np.ndarray:
        du, ds, lm = self.unpack(x)
        y1 = np.array([self.Fd[b] * du[b] + self.Aop(b, lm[b], adjoint=True) for b in range(self.B)])
        y2 = self.eps * ds - sum(self.PH_apply_re(b, lm[b]) for b in range(self.B))
        y3 = np.array([self.Aop(b, du[b]) - self.P_apply(b, ds) for b in range(self.B)])
        return self.pack(y1, y2, y3)

    def rhs(self) -> np.ndarray:
        b1 = fwi.scatter_weighted(self.prob, self.r)
        b2 = -self.eps * self.s_n / self.prob.gamma_ref if self.include_Ls_n else np.zeros(self.Nc)
        b3 = np.zeros((self.B, self.N), dtype=np.complex128)
        return self.pack(b1, b2, b3)

    def precond(self, v: np.ndarray, inner=None, inner_batch=None, hblock=None) -> np.ndarray:
        """z = P^{-1} v (eq. precond) or P~^{-1} v (eq. precond_approx) when
        ``inner(b, rhs, adjoint)`` approximates A'^{-1} / A'^{-H}.
        ``inner_batch(rhs [B, N], adjoint) -> [B, N]`` may replace the loop of
        per-block solves (the same solves, e.g. spread over processes).
        ``hblock(t) -> z_s`` replaces the H-block solve t / eps by another
        approximation of the reduced Hessian's inverse (Sec. 5 after eq.
        precond: e.g. L-BFGS, :mod:`oracle.lbfgs`)."""
        v1, v2, v3 = self.unpack(v)
        if inner_batch is None:
            if inner is None:
                def inner(b, rhs, adjoint):
                    return fwi.solve(self.prob, self.s_n, self.prob.block_freq(b), rhs, adjoint)

            def inner_batch(rhs, adjoint):
                return np.array([inner(b, rhs[b], adjoint) for b in range(self.B)])
        zl = inner_batch(v1, True)
        t = v2 + sum(self.PH_apply_re(b, zl[b]) for b in range(self.B))
        zs = t / self.eps if hblock is None else hblock(t)
        zu = inner_batch(np.array([v3[b] + self.P_apply(b, zs) for b in range(self.B)]), False)
        return self.pack(zu, zs, zl)

    def relres(self, x: np.ndarray) -> float:
        b = self.rhs()
        return float(np.linalg.norm(b - self.matvec(x)) / np.linalg.norm(b))

    def delta_s(self, x: np.ndarray) -> np.ndarray:
        """Model update in s^2/m^2: ds = gamma_ref * ds~."""
        return self.prob.gamma_ref * self.unpack(x)[1]

    # ---------------------------------------------------------------- direct references
    def real_form(self) -> sp.csr_matrix:
        """The whole scaled KKT matrix as a sparse real matrix in ``pack`` order."""
        I2 = sp.identity(2, format="csr")
        J2 = sp.csr_matrix(np.array([[0.0, -1.0], [1.0, 0.0]]))

        def realify(K):
            K = sp.csr_matrix(K)
            return sp.kron(K.real, I2) + sp.kron(K.imag, J2)

        B, N, Nc = self.B, self.N, self.Nc
        Ablk, AHblk, Fblk, Pr = [], [], [], []
        E = sp.csr_matrix((np.ones(Nc), (self.ci, np.arange(Nc))), shape=(N, Nc))
        for b in range(B):
            A = self.A[self.prob.block_freq(b)]
            Ablk.append(realify(A))
            AHblk.append(realify(A.conj().T))
            Fblk.append(sp.kron(sp.diags(self.Fd[b]), I2))
            # P~_b real form in interleaved order: rows 2n (re part), 2n+1 (im part)
            cP = (sp.diags(self.c[b]) @ E).tocoo()
            rows = np.concatenate([2 * cP.row, 2 * cP.row + 1])
            cols = np.concatenate([cP.col, cP.col])
            vals = np.concatenate([cP.data.real, cP.data.imag])
            Pr.append(sp.csr_matrix((vals, (rows, cols)), shape=(2 * N, Nc)))
        Fbig = sp.block_diag(Fblk)
        Abig = sp.block_diag(Ablk)
        AHbig = sp.block_diag(AHblk)
        Pbig = sp.vstack(Pr)
        Z = None
        M = sp.bmat([[Fbig, AHbig, Z],
                     [Abig, Z, -Pbig],
                     [Z, -Pbig.T, self.eps * sp.identity(Nc)]], format="csr")
        return M

    def solve_direct(self) -> np.ndarray:
        """Exact solution of the KKT system by sparse LU of the real form."""
        return spla.spsolve(self.real_form().tocsc(), self.rhs())

    def jacobian(self) -> list:
        """J~_b = Q_b A'^{-1} P~_b (dense, [R_b, Nc]) for every block."""
        Js = []
        for b in range(self.B):
            k = self.prob.block_src(b)
            ridx = H.receiver_indices(self.prob.grid, self.prob.survey, k)
            Qt = np.zeros((self.N, ridx.size), dtype=np.complex128)
            Qt[ridx, np.arange(ridx.size)] = 1.0
            lu = self.prob.lu(self.s_n, self.prob.block_freq(b))
            Y = lu.solve(Qt)                                      # A'^{-1} Q^T = (Q A'^{-1})^T
            Js.append((Y[self.ci, :] * self.c[b][self.ci][:, None]).T)
        return Js

    def normal_matvec(self, v: np.ndarray) -> np.ndarray:
        """H v without forming J (Sec. 3, eq. normal_system_discrete_sum, the
        form RSGN-CG uses): for every block one forward solve du = A'^{-1} P~ v
        and one adjoint solve lm = A'^{-H} F du, then eps v + sum Re(P~^H lm)."""
        out = self.eps * np.asarray(v, dtype=float).copy()
        for b in range(self.B):
            fi = self.prob.block_freq(b)
            du = fwi.solve(self.prob, self.s_n, fi, self.P_apply(b, v), False)
            lm = fwi.solve(self.prob, self.s_n, fi, self.Fd[b] * du, True)
            out += self.PH_apply_re(b, lm)
        return out

    def normal_rhs(self) -> np.ndarray:
        """g of the normal equations without forming J: one adjoint solve per
        block, g = sum Re(P~^H A'^{-H} Q^T W^2 r) - eps s_n/gamma_ref."""
        g = -self.eps * self.s_n / self.prob.gamma_ref if self.include_Ls_n else np.zeros(self.Nc)
        b1 = fwi.scatter_weighted(self.prob, self.r)
        for b in range(self.B):
            lm = fwi.solve(self.prob, self.s_n, self.prob.block_freq(b), b1[b], True)
            g = g + self.PH_apply_re(b, lm)
        return g

    def gn_lambda_max(self, iters: int):
        """Largest eigenvalue of the Gauss-Newton matrix G = Re(J~^H W^T W J~)
        (Sec. 3, eq. normal_system_discrete2 without eps I) by power iteration
        from the constant vector: v_0 = 1/||1||; w = G v_{k-1} (matrix-free:
        ``normal_matvec`` minus its eps v term); lambda_k = v_{k-1} . w;
        v_k = w / ||w||.  Returns [lambda_1, ..., lambda_iters]."""
        v = np.full(self.Nc, 1.0 / np.sqrt(self.Nc))
        out = []
        for _ in range(iters):
            w = self.normal_matvec(v) - self.eps * v
            out.append(float(v @ w))
            v = w / np.linalg.norm(w)
        return out

    def normal_system(self):
        """(H, g) of the reduced Gauss-Newton system (Sec. 3, eq.
        normal_system_discrete2) in the scaled control: H = sum Re(J^H W^2 J) + eps I,
        g = sum Re(J^H W^2 r) - eps s_n/gamma_ref."""
        Hm = self.eps * np.eye(self.Nc)
        g = -self.eps * self.s_n / self.prob.gamma_ref if self.include_Ls_n else np.zeros(self.Nc)
        for b, J in enumerate(self.jacobian()):
            w2 = H.receiver_weights(self.prob.survey, self.prob.block_src(b)) ** 2
            Hm += np.real(J.conj().T @ (w2[:, None] * J))
            g = g + np.real(J.conj().T @ (w2 * self.r[b]))
        return Hm, g
