"""Properties of the oracle's multigrid preconditioner and inner solver (a
design of its own for the shifted-Laplacian route named in Sec. 5).  The
cycle itself is pinned against its exact Fourier symbols in
test_oracle_mg_fourier, the BiCGStab iteration against scipy in
test_oracle_kkt.  CPU only."""
import numpy as np

import fwi_inputs as FI
from oracle import fwi, mg
from oracle import grid as G
from oracle import helmholtz as H


def _hier(nx=61, nz=41, npml=8, f=5.0, **kw):
    g = FI.Grid(nx=nx, nz=nz, npml=npml, h=20.0, pml_c=3000.0)
    v = FI.gradient_anomaly_model(nx, nz, seed=2)
    gp = G.pad_gamma(g, FI.gamma_of(v))
    return g, gp, mg.Hierarchy(g, 2 * np.pi * f, gp, **kw)


def test_prolongation_exact_for_linear_functions():
    """Bilinear interpolation reproduces a linear function at every fine node
    whose coarse neighbours exist (coarse node I sits on fine node 2I+1)."""
    g, gp, h = _hier()
    (nzf, nxf), (nzc, nxc) = h.shapes[0], h.shapes[1]
    J, I = np.meshgrid(np.arange(nzc), np.arange(nxc), indexing="ij")
    coarse = 3.0 + 0.5 * (2 * I + 1) - 0.25 * (2 * J + 1)
    fine = (h.P[0] @ coarse.ravel()).reshape(nzf, nxf)
    j, i = np.meshgrid(np.arange(nzf), np.arange(nxf), indexing="ij")
    expect = 3.0 + 0.5 * i - 0.25 * j
    inner = (i >= 1) & (j >= 1) & (i <= 2 * nxc - 1) & (j <= 2 * nzc - 1)
    np.testing.assert_allclose(fine[inner], expect[inner], rtol=1e-14)


def test_restriction_weights_sum_to_four():
    """R = P^T is 4x full weighting: interior coarse rows sum to 4."""
    g, gp, h = _hier()
    R = h.P[0].T.tocsr()
    sums = np.asarray(R.sum(axis=1)).ravel().reshape(h.shapes[1])
    np.testing.assert_allclose(sums[1:-1, 1:-1], 4.0)


def test_coarse_operators_are_rediscretisations():
    """Level-l operators equal the operator assembled directly on level l."""
    g, gp, h = _hier()
    for l in range(h.levels):
        A = H.assemble(g, 2 * np.pi * 5.0, H.level_gamma(g, gp, l), l, 0.5, sigma_cap=1.0)
        assert abs(A - h.ops[l]).max() == 0.0


def test_cycle_is_linear_and_jacobi_has_the_solution_as_fixed_point():
    g, gp, h = _hier()
    rng = np.random.default_rng(0)
    n = h.ops[0].shape[0]
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lhs = h.vcycle(2.0 * a - 3.0j * b)
    rhs = 2.0 * h.vcycle(a) - 3.0j * h.vcycle(b)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
    x = np.linalg.solve(h.ops[0].toarray(), a) if n < 3000 else None
    if x is not None:
        np.testing.assert_allclose(h.smooth(0, x, a, 3), x, rtol=1e-9, atol=1e-12)


def test_cycle_contracts_on_the_shifted_operator():
    """Used as a stationary iteration for M_beta x = b, the W(2,2) cycle reduces
    the residual by a factor < 0.8 per cycle (measured over 6 cycles)."""
    g, gp, h = _hier(nx=101, nz=61, npml=10)
    M = h.ops[0]
    b = np.random.default_rng(1).standard_normal(M.shape[0]) + 0j
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(6):
        x = x + h.vcycle(b - M @ x)
    factor = (np.linalg.norm(b - M @ x) / r0) ** (1 / 6)
    assert factor < 0.8, factor


def test_inner_solve_reduces_residual_and_adjoint_is_conjugate():
    """BiCGStab + multigrid reduces the residual of A' x = f; the adjoint solve
    equals conj(solve(conj f)) exactly (A'^H = conj(A'))."""
    wl = FI.tiny_workload()
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    s = wl.gamma_start.ravel()
    A = prob.operator(s, 0)
    hier = mg.Hierarchy(wl.grid, prob.omegas[0], prob.gamma_pad(s))
    f = H.source_vector(wl.grid, 50, 2, 1.0)
    x, hist = mg.inner_solve(A, hier, f, 30)
    assert hist[-1] < 1e-2, hist[-1]
    assert abs(np.linalg.norm(A @ x - f) / np.linalg.norm(f) - hist[-1]) < 1e-6
    rng = np.random.default_rng(2)
    v = rng.standard_normal(f.size) + 1j * rng.standard_normal(f.size)
    xa, _ = mg.inner_solve(A, hier, v, 5, adjoint=True)
    xb, _ = mg.inner_solve(A, hier, np.conj(v), 5)
    np.testing.assert_array_equal(xa, np.conj(xb))


def test_auto_levels():
    g = FI.Grid(nx=401, nz=141, npml=20, h=20.0)
    assert mg.auto_levels(g) == 6
    assert mg.level_shapes(g, 6)[-1] == (5, 13)
