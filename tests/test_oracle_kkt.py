"""Pins of the oracle's Gauss-Newton / KKT machinery (Sec. 3-5) against brute
force, finite differences and the invariants the paper states.  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.ndimage import gaussian_filter

import fwi_inputs as FI
from oracle import fwi, kkt, krylov
from oracle import helmholtz as H


def _micro(include=True, eps=1e-2, seed=0):
    wl = FI.micro_workload(seed=seed)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    return wl, prob, d, kkt.KKT(prob, wl.gamma_start.ravel(), d, eps, include_Ls_n=include)


def test_gradient_matches_central_differences():
    """Adjoint-state gradient (Sec. 3) against central differences of the misfit
    along smooth random directions (Gaussian-filtered noise)."""
    wl = FI.micro_workload(nx=25, nz=15)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    s0 = wl.gamma_start.ravel()
    phi, g = fwi.gradient(prob, s0, d)
    assert phi > 0
    for seed in range(4):
        rng = np.random.default_rng(seed)
        dirn = gaussian_filter(rng.standard_normal((wl.grid.nz, wl.grid.nx)), 2.0).ravel()
        dirn *= 0.01 * np.mean(s0) / np.abs(dirn).max()
        t = 1.0
        fp = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s0 + t * dirn), d))
        fm = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s0 - t * dirn), d))
        fd = (fp - fm) / (2 * t)
        an = float(np.dot(g, dirn))
        assert abs(fd - an) <= 1e-3 * abs(an), (seed, fd, an)


def test_taylor_remainder_second_order():
    wl = FI.micro_workload(nx=25, nz=15)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    s0 = wl.gamma_start.ravel()
    phi, g = fwi.gradient(prob, s0, d)
    dirn = gaussian_filter(np.random.default_rng(7).standard_normal((wl.grid.nz, wl.grid.nx)), 2.0).ravel()
    dirn *= 0.02 * np.mean(s0) / np.abs(dirn).max()
    rem = []
    for t in (1.0, 0.5, 0.25):
        f = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s0 + t * dirn), d))
        rem.append(abs(f - phi - t * np.dot(g, dirn)))
    assert 3.0 < rem[0] / rem[1] < 5.0 and 3.0 < rem[1] / rem[2] < 5.0, rem


def test_kkt_matrix_symmetric_and_matches_matvec():
    """eq. KKT is Hermitian (Sec. 4); with a real control its real form is a
    symmetric matrix, and the matrix-free product equals the assembled one."""
    _, _, _, K = _micro()
    M = K.real_form()
    assert abs(M - M.T).max() <= 1e-14 * abs(M).max()
    x = np.random.default_rng(3).standard_normal(K.size)
    np.testing.assert_allclose(K.matvec(x), M @ x, rtol=0, atol=1e-12 * np.abs(M @ x).max())


@pytest.mark.parametrize("include", [True, False])
def test_kkt_solution_equals_normal_equations(include):
    """Sec. 4, eqs. tmp1-normal_system_discrete3: eliminating du and lambda
    from the KKT system gives the reduced Gauss-Newton normal equations, so the
    two model updates coincide; du = A^{-1} P ds and lambda solves row 1."""
    _, prob, _, K = _micro(include=include)
    x = K.solve_direct()
    du, ds, lm = K.unpack(x)
    Hm, g = K.normal_system()
    ds_n = np.linalg.solve(Hm, g)
    assert np.linalg.norm(ds - ds_n) <= 1e-10 * np.linalg.norm(ds_n)
    for b in range(K.B):
        np.testing.assert_allclose(K.Aop(b, du[b]), K.P_apply(b, ds), atol=1e-10 * np.abs(du[b]).max())
    assert K.relres(x) < 1e-12


def test_exact_preconditioner_inverts_its_matrix():
    """P (eq. precond) applied to P^{-1} v returns v, with P assembled as the
    KKT matrix with its F block removed."""
    _, _, _, K = _micro()
    M = K.real_form().tolil()
    nU = 2 * K.B * K.N
    Fd = np.repeat(K.Fd.ravel(), 2)
    for i in np.nonzero(Fd)[0]:
        M[i, i] = M[i, i] - Fd[i]
    Pm = M.tocsr()
    v = np.random.default_rng(5).standard_normal(K.size)
    z = K.precond(v)
    assert np.linalg.norm(Pm @ z - v) <= 1e-10 * np.linalg.norm(v)
    assert nU > 0


def test_exact_preconditioner_gmres_iteration_bound():
    """M P^{-1} = I + diag(F, 0, 0) P^{-1}, so the preconditioned matrix minus
    the identity has rank <= rank(F) and GMRES with exact P converges in at
    most rank(F) + 1 iterations (Sec. 5; the U-factor remark of eq.
    permuted-block-LU).  Micro grid: 2 sources x 3 receivers -> rank(F) = 12."""
    _, _, _, K = _micro()
    rankF = 2 * int(np.count_nonzero(K.Fd))
    x, info = krylov.fgmres(K.matvec, K.rhs(), K.precond, restart=40, tol=1e-12, max_iter=40)
    assert info["iters"] <= rankF + 1, (info["iters"], rankF)
    assert info["true_relres"] < 1e-10


def test_zero_residual_gives_zero_update():
    """d = Q S(s_n) and no -L s_n term: r = 0 so b = 0 and ds = 0 exactly."""
    wl = FI.micro_workload()
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    s = wl.gamma_start.ravel()
    d = fwi.sample(prob, fwi.forward(prob, s))
    K = kkt.KKT(prob, s, d, 1e-2, include_Ls_n=False)
    assert np.abs(K.rhs()).max() < 1e-14 * 1e3
    x, info = krylov.fgmres(K.matvec, K.rhs(), K.precond)
    assert np.all(K.unpack(x)[1] == 0.0)


def test_fgmres_matches_direct_solve_tiny():
    """The tiny workload (101x51, 4 sources, 5 Hz): GMRES with the exact
    preconditioner (the paper's GMRes-full) reaches 1e-8 and its model update
    matches the sparse direct solve of the whole KKT system."""
    wl = FI.tiny_workload()
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    x, info = krylov.fgmres(K.matvec, K.rhs(), K.precond, restart=30, tol=1e-8, max_iter=300)
    assert info["true_relres"] <= 1e-8
    xd = K.solve_direct()
    ds, dsd = K.unpack(x)[1], K.unpack(xd)[1]
    assert np.linalg.norm(ds - dsd) <= 1e-6 * np.linalg.norm(dsd)


def test_fgmres_and_bicgstab_on_small_dense_systems():
    """The Krylov routines against numpy.linalg.solve (library routine)."""
    rng = np.random.default_rng(11)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, info = krylov.fgmres(lambda v: A @ v, b, restart=10, tol=1e-12, max_iter=400)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)
    Ac = A + 1j * rng.standard_normal((n, n)) * 0.2
    bc = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    M = np.diag(1 / np.diag(Ac))
    xc, hist = krylov.bicgstab(lambda v: Ac @ v, bc, lambda v: M @ v, iters=200, tol=1e-13)
    np.testing.assert_allclose(xc, np.linalg.solve(Ac, bc), rtol=1e-9, atol=1e-10)


def test_newton_step_reduces_misfit():
    """Sanity (not a pin): one full Gauss-Newton step lowers the misfit."""
    wl, prob, d, K = _micro(include=False, eps=1e-3)
    x = K.solve_direct()
    s1 = K.s_n + K.delta_s(x)
    phi0 = fwi.misfit(prob, K.r)
    phi1 = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s1), d))
    assert phi1 < phi0


def test_cg_on_small_spd_systems():
    """Conjugate gradients (the Krylov method of RSGN-CG, Sec. 3) against a dense
    solve; in exact arithmetic CG ends within n iterations, so on a 40 x 40 SPD
    system with a spread spectrum it reaches 1e-12 within a few more."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    Hm = Q @ np.diag(np.logspace(0, 2, 40)) @ Q.T
    g = rng.standard_normal(40)
    x, hist = krylov.cg(lambda v: Hm @ v, g, tol=1e-12, max_iter=200)
    assert np.linalg.norm(x - np.linalg.solve(Hm, g)) <= 1e-10 * np.linalg.norm(x)
    assert len(hist) <= 60 and hist[-1] <= 1e-12
    # an identity-plus-rank-3 matrix is solved in at most 4 iterations
    U = rng.standard_normal((40, 3))
    H2 = np.eye(40) + U @ U.T
    _, h2 = krylov.cg(lambda v: H2 @ v, g, tol=1e-10, max_iter=50)
    assert len(h2) <= 4


def test_matrix_free_normal_operator_equals_the_dense_normal_system():
    """The forward/adjoint-solve form of H v and g (what RSGN-CG applies, one
    forward and one adjoint solve per block) equals the explicit
    J^H W^2 J + eps I built column by column."""
    _, _, _, K = _micro()
    Hm, g = K.normal_system()
    rng = np.random.default_rng(4)
    for _ in range(2):
        v = rng.standard_normal(K.Nc)
        hv = K.normal_matvec(v)
        assert np.linalg.norm(hv - Hm @ v) <= 1e-10 * np.linalg.norm(Hm @ v)
    assert np.linalg.norm(K.normal_rhs() - g) <= 1e-10 * np.linalg.norm(g)


def test_rsgn_cg_reaches_the_kkt_update():
    """RSGN-CG (Sec. 3) and the full-space KKT system give the same, unique
    update (eps > 0): CG on the matrix-free normal operator against the sparse
    direct solve of the KKT system."""
    _, _, _, K = _micro()
    ds_cg, hist = krylov.cg(K.normal_matvec, K.normal_rhs(), tol=1e-12, max_iter=200)
    ds_kkt = K.unpack(K.solve_direct())[1]
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(ds_cg - ds_kkt) <= 1e-8 * np.linalg.norm(ds_kkt)


@pytest.mark.parametrize("with_precond", [False, True])
def test_bicgstab_iterates_equal_scipy(with_precond):
    """The inner solver's fixed-iteration form (k iterations from x = 0, shadow
    residual b, right preconditioning) is van der Vorst's BiCGStab, iterate by
    iterate: after k iterations it equals scipy.sparse.linalg.bicgstab stopped
    at maxiter = k, on a complex non-Hermitian system, with and without a
    (Jacobi) preconditioner."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(12)
    n = 80
    A = (np.eye(n) * (3 + 1j) + rng.standard_normal((n, n)) * 0.25
         + 1j * rng.standard_normal((n, n)) * 0.15)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Minv = np.diag(1 / np.diag(A))
    pre = (lambda v: Minv @ v) if with_precond else None
    Mop = spla.LinearOperator((n, n), matvec=lambda v: Minv @ v, dtype=complex) if with_precond else None
    for k in (1, 2, 5, 9):
        x, _ = krylov.bicgstab(lambda v: A @ v, b, pre, iters=k, tol=0.0)
        xs, _ = spla.bicgstab(A, b, rtol=1e-300, atol=0.0, maxiter=k, M=Mop)
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs), (k, np.linalg.norm(x - xs))


def _weighted_micro(seed=0, nx=21, nz=13, eps=1e-2, include=True):
    """Micro workload whose data weights W are not all 1 (uniform in [0.5, 2])."""
    wl = FI.micro_workload(seed=seed, nx=nx, nz=nz, n_rec=5)
    wl.survey.rec_w = np.random.default_rng(100 + seed).uniform(0.5, 2.0, wl.survey.rec_w.shape)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    return wl, prob, d, kkt.KKT(prob, wl.gamma_start.ravel(), d, eps, include_Ls_n=include)


def test_coupling_block_by_finite_differences_of_the_data():
    """The coupling P~_b = h^2 gamma_ref omega_b^2 diag(u_b) E of the scaled KKT
    system (Sec. 3, eq. P; Sec. 4) is the derivative of the state equation with
    respect to the scaled control: the linearised data J~_b ds~ = Q A'^{-1} P~_b ds~
    must equal the central difference of the forward data,
    (Q u(s + t gamma_ref ds~) - Q u(s - t gamma_ref ds~)) / 2t.  A wrong factor
    (h^2, gamma_ref, omega^2), a conjugate or a sign in P~ fails this."""
    wl, prob, d, K = _weighted_micro(nx=25, nz=15)
    s0 = K.s_n
    rng = np.random.default_rng(21)
    dst = gaussian_filter(rng.standard_normal((wl.grid.nz, wl.grid.nx)), 2.0).ravel()
    dst /= np.abs(dst).max()                       # ds~ = O(1): ds = gamma_ref ds~
    t = 1e-4
    qp = fwi.sample(prob, fwi.forward(prob, s0 + t * prob.gamma_ref * dst))
    qm = fwi.sample(prob, fwi.forward(prob, s0 - t * prob.gamma_ref * dst))
    Js = K.jacobian()
    for b in range(K.B):
        fd = (qp[b] - qm[b]) / (2 * t)
        lin = Js[b] @ dst
        du = fwi.solve(prob, s0, prob.block_freq(b), K.P_apply(b, dst))
        q_lin = du[H.receiver_indices(wl.grid, wl.survey, prob.block_src(b))]
        assert np.linalg.norm(lin - fd) <= 1e-6 * np.linalg.norm(fd), (b, np.linalg.norm(lin - fd) / np.linalg.norm(fd))
        assert np.linalg.norm(q_lin - fd) <= 1e-6 * np.linalg.norm(fd)


def test_weighted_gradient_matches_central_differences():
    """W != 1 (Sec. 3: Phi = 1/2 ||W r||^2): the adjoint gradient, whose adjoint
    source is Q^T W^T W r, against central differences of the weighted misfit."""
    wl, prob, d, K = _weighted_micro(nx=25, nz=15)
    s0 = K.s_n
    phi, g = fwi.gradient(prob, s0, d)
    for seed in range(3):
        dirn = gaussian_filter(np.random.default_rng(seed).standard_normal((wl.grid.nz, wl.grid.nx)), 2.0).ravel()
        dirn *= 0.01 * np.mean(s0) / np.abs(dirn).max()
        fp = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s0 + dirn), d))
        fm = fwi.misfit(prob, fwi.residual(prob, fwi.forward(prob, s0 - dirn), d))
        an = float(np.dot(g, dirn))
        assert abs((fp - fm) / 2 - an) <= 1e-3 * abs(an), (seed, (fp - fm) / 2, an)


def test_weighted_misfit_and_gradient_scale_with_w_squared():
    """Multiplying every weight by 3 multiplies the misfit and its gradient by 9
    (W enters squared); a single W in place of W^T W would give 3."""
    wl, prob, d, K = _weighted_micro()
    s0 = K.s_n
    phi1, g1 = fwi.gradient(prob, s0, d)
    wl.survey.rec_w = 3.0 * wl.survey.rec_w
    prob3 = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    phi3, g3 = fwi.gradient(prob3, s0, d)
    assert abs(phi3 - 9 * phi1) <= 1e-12 * phi3
    assert np.linalg.norm(g3 - 9 * g1) <= 1e-11 * np.linalg.norm(g3)
    direct = 0.5 * sum(float(np.sum((w * np.abs(rb)) ** 2)) for w, rb in
                       zip([wl.survey.rec_w[wl.survey.rec_offsets[prob.block_src(b)]:
                                            wl.survey.rec_offsets[prob.block_src(b) + 1]]
                            for b in range(prob.n_blocks)], K.r))
    assert abs(phi3 - direct) <= 1e-12 * direct


@pytest.mark.parametrize("include", [True, False])
def test_weighted_kkt_update_is_the_weighted_least_squares_solution(include):
    """With W != 1 the KKT update (Sec. 4) is the minimiser of the linearised
    problem 1/2 ||W (r - J~ ds~)||^2 + eps/2 ||s_n/gamma_ref + ds~||^2 (Sec. 3),
    computed here by numpy.linalg.lstsq on the stacked real system
    [W J~; sqrt(eps) I] ds~ = [W r; -sqrt(eps) s_n/gamma_ref] (row scaling by W,
    not the W^2 of the normal equations and of F = Q^T W^T W Q)."""
    wl, prob, d, K = _weighted_micro(include=include)
    rows, rhs = [], []
    for b, J in enumerate(K.jacobian()):
        w = H.receiver_weights(wl.survey, prob.block_src(b))
        WJ, Wr = w[:, None] * J, w * K.r[b]
        rows += [WJ.real, WJ.imag]
        rhs += [Wr.real, Wr.imag]
    se = np.sqrt(K.eps)
    rows.append(se * np.eye(K.Nc))
    rhs.append(-se * K.s_n / prob.gamma_ref if include else np.zeros(K.Nc))
    ds_ls = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
    ds_kkt = K.unpack(K.solve_direct())[1]
    assert np.linalg.norm(ds_kkt - ds_ls) <= 1e-8 * np.linalg.norm(ds_ls)


def test_gauss_newton_lambda_max_by_power_iteration():
    """The regulariser rule eps = alpha * lambda_max(Re J~^H W^2 J~) needs the
    largest eigenvalue of the Gauss-Newton matrix (Sec. 3).  The power
    iteration's Rayleigh quotients never exceed it, never decrease (G is
    symmetric positive semidefinite) and converge to numpy.linalg.eigvalsh of
    the dense matrix built column by column."""
    _, _, _, K = _weighted_micro()
    Hm, _ = K.normal_system()
    G = Hm - K.eps * np.eye(K.Nc)
    lmax = np.linalg.eigvalsh(G).max()
    lam = K.gn_lambda_max(60)
    assert all(l <= lmax * (1 + 1e-12) for l in lam)
    assert all(b >= a * (1 - 1e-12) for a, b in zip(lam, lam[1:]))
    assert abs(lam[-1] - lmax) <= 1e-6 * lmax, (lam[-1], lmax)
