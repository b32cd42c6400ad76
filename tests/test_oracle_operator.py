"""Pins of the oracle's Helmholtz operator (Sec. 2) against closed forms,
library routines and invariants.  CPU only."""
from dataclasses import replace

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import hankel1

import fwi_inputs as FI
from oracle import grid as G
from oracle import helmholtz as H


def _grid(nx=21, nz=17, npml=5, h=10.0, **kw):
    return FI.Grid(nx=nx, nz=nz, npml=npml, h=h, **kw)


def test_no_layer_is_negative_laplacian_minus_mass():
    """Sec. 2: without the layer, A = -Delta - omega^2 diag(gamma) (real
    symmetric indefinite); compare with the 5-point Laplacian assembled from
    scipy Kronecker products."""
    g = _grid(npml=0)
    rng = np.random.default_rng(1)
    gam = 1.0 / rng.uniform(1500, 3000, size=(g.nz, g.nx)) ** 2
    om = 2 * np.pi * 7.0
    A = H.assemble(g, om, gam, scaled=False)
    def T(n):
        return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1])
    lap = (sp.kron(sp.identity(g.nz), T(g.nx)) + sp.kron(T(g.nz), sp.identity(g.nx))) / g.h ** 2
    ref = -lap - om ** 2 * sp.diags(gam.ravel())
    assert abs(A - ref).max() < 1e-12 * abs(ref).max()
    assert abs(A.imag).max() == 0.0


@pytest.mark.parametrize("level,shift", [(0, 0.0), (0, 0.5), (1, 0.5), (2, 0.5)])
def test_operator_is_complex_symmetric(level, shift):
    """A^T = A exactly, so A^H = conj(A): the adjoint solve is the forward
    solve on conjugated data (used by both the oracle and the CUDA path)."""
    g = _grid(nx=31, nz=23)
    gam = G.pad_gamma(g, np.full((g.nz, g.nx), 1 / 2000.0 ** 2))
    from oracle.helmholtz import level_gamma
    A = H.assemble(g, 2 * np.pi * 5, level_gamma(g, gam, level), level, shift)
    assert abs(A - A.T).max() == 0.0
    assert A.shape[0] > 0


def test_layer_damps_and_is_nontrivial():
    g = _grid()
    pa = G.stretch_arrays(g, 2 * np.pi * 5)
    X = pa["X"]
    assert np.all(X.real == 1.0)
    assert X.imag[0] > 0 and X.imag[g.npml] == 0.0 and X.imag[-1] > 0
    # profile is quadratic in the distance into the layer
    d = np.arange(g.npml, 0, -1) * g.h
    np.testing.assert_allclose(X.imag[:g.npml], G.sigma_max(g) * (d / (g.npml * g.h)) ** 2 / (2 * np.pi * 5))


def _point_source_field(n_core, npml, h, c, f):
    g = FI.Grid(nx=n_core, nz=n_core, npml=npml, h=h, pml_c=c, pml_R=1e-3)
    Nz, Nx = G.padded_shape(g)
    gam = np.full((Nz, Nx), 1.0 / c ** 2)
    A = H.assemble(g, 2 * np.pi * f, gam, scaled=False)
    src = n_core // 2
    rhs = np.zeros(Nz * Nx, dtype=complex)
    rhs[G.padded_index(g, src, src)] = 1.0 / h ** 2          # unit discrete delta
    u = spla.spsolve(A.tocsc(), rhs).reshape(Nz, Nx)
    return g, u, src


def test_green_function_hankel_second_order():
    """Closed form: in a homogeneous medium the field of a unit point source is
    (i/4) H0^(1)(k r) (time convention e^{-i omega t}, outgoing); the 5-point
    scheme converges at second order.  Compare on the same physical ring
    (r between 100 and 300 m) at h and h/2."""
    c, f = 2000.0, 10.0
    k = 2 * np.pi * f / c
    errs = []
    for h, n, p in ((10.0, 81, 30), (5.0, 161, 60)):
        g, u, s = _point_source_field(n, p, h, c, f)
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        r = h * np.hypot(ii - s, jj - s)
        ring = (r >= 100.0) & (r <= 300.0)
        core = u[p:p + n, p:p + n]
        ref = 0.25j * hankel1(0, k * r[ring])
        errs.append(np.linalg.norm(core[ring] - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.05, errs
    assert errs[1] < 0.015, errs
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


def test_layer_reflection_small():
    """The absorbing layer: the field inside the core of a small padded domain
    agrees with the field of a domain three times wider to well under 1 %."""
    c, f, h = 2000.0, 10.0, 10.0
    _, u1, s1 = _point_source_field(61, 20, h, c, f)
    g3, u3, s3 = _point_source_field(181, 20, h, c, f)
    c1 = u1[20:81, 20:81]
    c3 = u3[20 + 60:20 + 121, 20 + 60:20 + 121]
    rel = np.linalg.norm(c1 - c3) / np.linalg.norm(c3)
    assert rel < 0.01, rel


def test_reciprocity():
    """Green's functions are reciprocal (A^T = A): u_s(x_r) = u_r(x_s)."""
    wl = FI.micro_workload()
    g = wl.grid
    from oracle import fwi
    prob = fwi.Problem.create(g, wl.survey, wl.gamma_start)
    A = prob.operator(wl.gamma_start.ravel(), 0)
    a = G.padded_index(g, 2, 3)
    b = G.padded_index(g, 11, 8)
    ea = np.zeros(A.shape[0], complex); ea[a] = 1
    eb = np.zeros(A.shape[0], complex); eb[b] = 1
    ua = spla.spsolve(A.tocsc(), ea)
    ub = spla.spsolve(A.tocsc(), eb)
    assert abs(ua[b] - ub[a]) < 1e-12 * abs(ua[b])


def test_lu_residual():
    wl = FI.tiny_workload()
    from oracle import fwi
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    s = wl.gamma_start.ravel()
    u = fwi.forward(prob, s)
    A = prob.operator(s, 0)
    for b in range(prob.n_blocks):
        f = H.source_vector(wl.grid, int(wl.survey.src_ix[b]), int(wl.survey.src_iz[b]), 1.0)
        assert np.linalg.norm(A @ u[b] - f) <= 1e-12 * np.linalg.norm(f)


def test_level_gamma_constant_and_mean():
    """Normalised full weighting keeps a constant model constant and a linear
    model linear away from the edges."""
    g = _grid(nx=41, nz=31)
    Nz, Nx = G.padded_shape(g)
    assert np.allclose(H.level_gamma(g, np.full((Nz, Nx), 3.0), 2), 3.0)
    lin = np.add.outer(np.arange(Nz), 2.0 * np.arange(Nx))
    c1 = H.level_gamma(g, lin, 1)
    J, I = np.meshgrid(np.arange(c1.shape[0]), np.arange(c1.shape[1]), indexing="ij")
    expect = (2 * J + 1) + 2.0 * (2 * I + 1)
    inner = (J > 0) & (I > 0) & (J < c1.shape[0] - 1) & (I < c1.shape[1] - 1)
    np.testing.assert_allclose(c1[inner], expect[inner])
