"""Pins of the oracle's L-BFGS H block (oracle/lbfgs.py) and of its place in
the preconditioner (Sec. 5 after eq. precond: H ~ L, or another
approximation of the reduced Hessian such as L-BFGS).

* Quadratic termination and the hereditary property: BFGS with exact line
  searches on a strictly convex quadratic f(x) = x^T A x / 2 - c^T x reaches the
  minimiser A^{-1} c in n steps, and every stored pair satisfies
  B^{-1} y_j = s_j (Nocedal & Wright, Theorem 6.4 context: conjugate
  directions).  The two-loop recursion is the inverse-Hessian product of that
  run, so a wrong sign, order or scaling in it breaks the termination.
* Spectral closed form: pairs (v_j, lambda_j v_j) of orthonormal eigenvectors
  of an SPD matrix give B^{-1} = h0 (I - V V^T) + V diag(1/lambda) V^T.
* Secant equation for the newest pair; symmetry and positive definiteness of
  the matrix assembled column by column; the matrix update formula agrees.
* The preconditioner: with the exact reduced Hessian in the H block (exact
  block solves), the preconditioned KKT matrix satisfies (P^{-1} M - I)^2 = 0,
  so FGMRES stops after 2 iterations at any eps; the same holds with L-BFGS
  built from all eigenpairs of the reduced Hessian, and with no pairs the
  block is the paper's L = eps I.
"""
import numpy as np
import pytest

import fwi_inputs as FI
from oracle import fwi, kkt, krylov, lbfgs


def _spd(n, seed, cond=50.0):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T, Q, lam


@pytest.mark.parametrize("h0", [1.0, 0.05, 3.0])
def test_bfgs_quadratic_termination_and_hereditary_property(h0):
    n = 9
    A, _, _ = _spd(n, 1)
    c = np.random.default_rng(2).standard_normal(n)
    x = np.zeros(n)
    pairs = []
    for k in range(n):
        grad = A @ x - c
        if np.linalg.norm(grad) < 1e-13:
            break
        p = -lbfgs.two_loop(grad, pairs, h0)
        t = -(grad @ p) / (p @ A @ p)                 # exact line search
        s = t * p
        x = x + s
        pairs.append((s, A @ s))
        for sj, yj in pairs:                          # hereditary: B^{-1} y_j = s_j
            np.testing.assert_allclose(lbfgs.two_loop(yj, pairs, h0), sj, rtol=1e-8, atol=1e-10 * np.linalg.norm(sj))
    np.testing.assert_allclose(x, np.linalg.solve(A, c), rtol=1e-9)


def test_spectral_pairs_give_the_closed_form():
    n, m, h0 = 12, 5, 0.3
    A, Q, lam = _spd(n, 3)
    V = Q[:, :m]
    pairs = [(V[:, j] * 2.0, A @ (V[:, j] * 2.0)) for j in range(m)]   # any scaling of the eigenvectors
    Binv = h0 * (np.eye(n) - V @ V.T) + (V / lam[:m]) @ V.T
    q = np.random.default_rng(4).standard_normal(n)
    np.testing.assert_allclose(lbfgs.two_loop(q, pairs, h0), Binv @ q, rtol=1e-12)
    # all n eigenpairs: the exact inverse
    full = [(Q[:, j], A @ Q[:, j]) for j in range(n)]
    np.testing.assert_allclose(lbfgs.two_loop(q, full, h0), np.linalg.solve(A, q), rtol=1e-11)


def test_secant_symmetry_definiteness_and_matrix_form():
    n, h0 = 10, 0.7
    g = np.random.default_rng(5)
    A, _, _ = _spd(n, 6)
    pairs = []
    for _ in range(4):
        s = g.standard_normal(n)
        pairs.append((s, A @ s))
    s_new, y_new = pairs[-1]
    np.testing.assert_allclose(lbfgs.two_loop(y_new, pairs, h0), s_new, rtol=1e-11)
    Bm = np.column_stack([lbfgs.two_loop(e, pairs, h0) for e in np.eye(n)])
    np.testing.assert_allclose(Bm, Bm.T, atol=1e-12 * np.abs(Bm).max())
    assert np.linalg.eigvalsh((Bm + Bm.T) / 2).min() > 0
    np.testing.assert_allclose(Bm, lbfgs.dense_inverse(pairs, h0, n), rtol=1e-10, atol=1e-13)
    # no pairs: H_0 itself
    np.testing.assert_allclose(lbfgs.two_loop(g.standard_normal(n) * 0 + 1.0, [], h0), np.full(n, h0))


def test_pairs_without_curvature_are_refused():
    s = np.array([1.0, 0.0])
    with pytest.raises(ValueError):
        lbfgs.two_loop(s, [(s, -s)], 1.0)


@pytest.fixture(scope="module")
def micro():
    wl = FI.micro_workload()
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    return wl, prob, d


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-5])
def test_exact_hessian_block_converges_in_two_iterations(micro, eps):
    wl, prob, d = micro
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, eps)
    Hm, _ = K.normal_system()
    Hinv = np.linalg.inv(Hm)
    x, info = krylov.fgmres(K.matvec, K.rhs(), lambda v: K.precond(v, hblock=lambda t: Hinv @ t),
                            restart=30, tol=1e-10, max_iter=50)
    assert info["iters"] <= 2 and info["true_relres"] <= 1e-10
    np.testing.assert_allclose(K.delta_s(x), K.delta_s(K.solve_direct()), rtol=1e-8, atol=1e-14)
    # L-BFGS from every eigenpair of the reduced Hessian is the same block
    lam, Q = np.linalg.eigh(Hm)
    pairs = [(Q[:, j], Hm @ Q[:, j]) for j in range(K.Nc)]
    x2, info2 = krylov.fgmres(K.matvec, K.rhs(),
                              lambda v: K.precond(v, hblock=lambda t: lbfgs.two_loop(t, pairs, 1.0 / eps)),
                              restart=30, tol=1e-10, max_iter=50)
    assert info2["iters"] <= 2
    # no pairs: the paper's L = eps I (same iterates as the default block)
    z0 = K.precond(K.rhs())
    z1 = K.precond(K.rhs(), hblock=lambda t: lbfgs.two_loop(t, [], 1.0 / eps))
    np.testing.assert_allclose(z1, z0, rtol=1e-12, atol=1e-14 * np.abs(z0).max())
