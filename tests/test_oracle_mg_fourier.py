"""Pins of the oracle's multigrid cycle by exact Fourier (sine-mode) analysis.

The paper names the shifted-Laplacian preconditioner with multigrid as the
inner block solver (Sec. 5, after eq. precond_approx) and leaves its parts
open; the oracle's cycle (oracle/mg.py) is pinned here against an independent
closed form rather than against itself.

On a grid without the absorbing layer, with constant gamma and n = 2^k - 1
nodes per direction on the fine level (so every coarser level again has
2^(k-l) - 1 nodes and coarse node I sits on fine node 2I+1), the h_l^2-scaled
shifted operator  M_l = -h_l^2 Delta_h - (1 + i beta)(omega h_l)^2 gamma
with Dirichlet ghosts is diagonalised by the sine modes
    v_pq[j, i] = sin(p pi (i+1)/(nx+1)) sin(q pi (j+1)/(nz+1)),
with eigenvalue  (2 - 2 cos t_p) + (2 - 2 cos t_q) - c_l,  t_p = p pi/(nx+1).
Its diagonal is the constant 4 - c_l, so damped Jacobi multiplies v_pq by
1 - w lambda_pq / (4 - c_l).  Per direction, restriction by R = P^T maps
fine mode p (p <= n_c) to coarse mode p times (1 + cos t_p) and fine mode
n+1-p to coarse mode p times -(1 - cos t_p); fine mode n_c + 1 maps to zero.
Bilinear prolongation maps coarse mode p to (1 + cos t_p)/2 fine mode p plus
(cos t_p - 1)/2 fine mode n+1-p.  These are the textbook one-dimensional
symbols (e.g. Trottenberg, Oosterlee & Schueller, Multigrid, 2001, ch. 4)
in product form.

The cycle is then evaluated mode by mode (a function of one level is a
dictionary {(p, q): coefficient}) and compared with ``Hierarchy.vcycle``
applied to the synthesised grid functions.  A wrong Jacobi diagonal, damping
or sweep count, a transposed or mis-weighted transfer, a wrong coarse-level
spacing in the mass term, or a wrong W/V recursion depth changes the result
far beyond the 1e-12 tolerance (the last test shows that the comparison
separates V from W).  CPU only."""
import numpy as np
import pytest

import fwi_inputs as FI
from oracle import grid as G
from oracle import mg

BETA = 0.5
GAMMA = 1.0 / 2000.0 ** 2


def _sizes(n0: int, levels: int):
    out = [n0]
    for _ in range(levels - 1):
        out.append(out[-1] // 2)
    return out


class Symbol:
    """The multigrid cycle of the shifted operator on sine-mode coefficients."""

    def __init__(self, nx, nz, levels, h, omega, nu1=2, nu2=2, wj=0.5, cycle=2, wdepth=2):
        self.nx, self.nz = _sizes(nx, levels), _sizes(nz, levels)
        self.levels = levels
        self.c = [(1.0 + 1j * BETA) * (omega * h * 2 ** l) ** 2 * GAMMA for l in range(levels)]
        self.nu1, self.nu2, self.wj, self.cycle, self.wdepth = nu1, nu2, wj, cycle, wdepth

    def lam(self, l, p, q):
        tp = np.pi * p / (self.nx[l] + 1)
        tq = np.pi * q / (self.nz[l] + 1)
        return (2.0 - 2.0 * np.cos(tp)) + (2.0 - 2.0 * np.cos(tq)) - self.c[l]

    def apply_M(self, l, v):
        return {k: a * self.lam(l, *k) for k, a in v.items()}

    def smooth(self, l, x, b, sweeps):
        d = 4.0 - self.c[l]
        keys = set(x) | set(b)
        for _ in range(sweeps):
            x = {k: x.get(k, 0.0) + self.wj * (b.get(k, 0.0) - x.get(k, 0.0) * self.lam(l, *k)) / d
                 for k in keys}
        return x

    @staticmethod
    def _r1(p, n):
        """(coarse mode, factor) of fine mode p under 1D restriction, or None."""
        nc = (n - 1) // 2
        t = np.pi * p / (n + 1)
        if p <= nc:
            return p, 1.0 + np.cos(t)
        if p == nc + 1:
            return None
        return n + 1 - p, -(1.0 + np.cos(t))

    def restrict(self, l, v):
        out = {}
        for (p, q), a in v.items():
            rx, rz = self._r1(p, self.nx[l]), self._r1(q, self.nz[l])
            if rx is None or rz is None:
                continue
            k = (rx[0], rz[0])
            out[k] = out.get(k, 0.0) + a * rx[1] * rz[1]
        return out

    @staticmethod
    def _p1(p, n):
        t = np.pi * p / (n + 1)
        return [(p, 0.5 * (1.0 + np.cos(t))), (n + 1 - p, 0.5 * (np.cos(t) - 1.0))]

    def prolong(self, l, v):
        out = {}
        for (p, q), a in v.items():
            for fp, wx in self._p1(p, self.nx[l]):
                for fq, wz in self._p1(q, self.nz[l]):
                    out[(fp, fq)] = out.get((fp, fq), 0.0) + a * wx * wz
        return out

    def cycle_from_zero(self, b, l=0):
        if l == self.levels - 1:
            return {k: a / self.lam(l, *k) for k, a in b.items()}
        x = self.smooth(l, {}, b, self.nu1)
        for _ in range(self.cycle if 0 < l <= self.wdepth else 1):
            Mx = self.apply_M(l, x)
            r = {k: b.get(k, 0.0) - Mx.get(k, 0.0) for k in set(b) | set(Mx)}
            e = self.prolong(l, self.cycle_from_zero(self.restrict(l, r), l + 1))
            x = {k: x.get(k, 0.0) + e.get(k, 0.0) for k in set(x) | set(e)}
        return self.smooth(l, x, b, self.nu2)


def _sine(n):
    idx = np.arange(1, n + 1)
    return np.sin(np.pi * np.outer(idx, idx) / (n + 1))        # [mode p-1, node i]


def _synth(coef: dict, nx, nz):
    C = np.zeros((nz, nx), dtype=np.complex128)
    for (p, q), a in coef.items():
        C[q - 1, p - 1] += a
    return (_sine(nz).T @ C @ _sine(nx)).ravel()               # [j, i] = sum C[q,p] S_z[q,j] S_x[p,i]


def _hier(nx, nz, levels, f=5.0, h=20.0, **kw):
    g = FI.Grid(nx=nx, nz=nz, npml=0, h=h)
    gp = np.full((nz, nx), GAMMA)
    return mg.Hierarchy(g, 2 * np.pi * f, gp, shift=BETA, levels=levels, **kw)


def _random_coef(nx, nz, seed):
    rng = np.random.default_rng(seed)
    return {(p, q): complex(rng.standard_normal(), rng.standard_normal())
            for p in range(1, nx + 1) for q in range(1, nz + 1)}


@pytest.mark.parametrize("levels,wdepth,cycle,nu", [
    (2, 2, 2, (2, 2)),        # two-grid, exact coarse solve
    (3, 2, 2, (2, 2)),        # W on level 1
    (4, 1, 2, (2, 2)),        # W on level 1, V on level 2
    (4, 2, 2, (1, 3)),        # W on levels 1-2, uneven sweeps
    (3, 2, 1, (2, 2)),        # V throughout
])
def test_cycle_equals_fourier_symbol(levels, wdepth, cycle, nu):
    nx, nz, f, h = 31, 15, 5.0, 20.0
    hier = _hier(nx, nz, levels, f, h, nu1=nu[0], nu2=nu[1], wj=0.5, cycle=cycle, wdepth=wdepth)
    assert hier.shapes[0] == (nz, nx) and hier.shapes[-1] == (_sizes(nz, levels)[-1], _sizes(nx, levels)[-1])
    sym = Symbol(nx, nz, levels, h, 2 * np.pi * f, nu1=nu[0], nu2=nu[1], wj=0.5, cycle=cycle, wdepth=wdepth)
    b = _random_coef(nx, nz, seed=levels)
    x_oracle = hier.vcycle(_synth(b, nx, nz))
    x_symbol = _synth(sym.cycle_from_zero(b), nx, nz)
    err = np.linalg.norm(x_oracle - x_symbol) / np.linalg.norm(x_symbol)
    assert err <= 1e-12, err


def test_two_grid_error_operator_on_one_harmonic_quadruple():
    """The two-grid error operator E = S^nu2 (I - P M_c^{-1} R M) S^nu1 maps the
    four harmonics {(p,q), (n+1-p,q), (p,n+1-q), (n+1-p,n+1-q)} of one coarse
    mode onto themselves; the oracle's E applied to (p,q) has no component
    outside them and equals the 4x4 symbol built from the closed-form factors."""
    nx, nz, f, h = 31, 15, 5.0, 20.0
    hier = _hier(nx, nz, 2, f, h)
    M = hier.ops[0]
    sym = Symbol(nx, nz, 2, h, 2 * np.pi * f)
    p, q = 5, 3
    v = _synth({(p, q): 1.0}, nx, nz)
    Ev = v - hier.vcycle(M @ v)
    # closed form: smoothing factors, transfer factors, coarse eigenvalue
    fam = [(p, q), (nx + 1 - p, q), (p, nz + 1 - q), (nx + 1 - p, nz + 1 - q)]
    d0 = 4.0 - sym.c[0]
    s = {k: 1.0 - 0.5 * sym.lam(0, *k) / d0 for k in fam}
    tp, tq = np.pi * p / (nx + 1), np.pi * q / (nz + 1)
    rx = {p: 1 + np.cos(tp), nx + 1 - p: -(1 - np.cos(tp))}
    rz = {q: 1 + np.cos(tq), nz + 1 - q: -(1 - np.cos(tq))}
    px = {p: (1 + np.cos(tp)) / 2, nx + 1 - p: (np.cos(tp) - 1) / 2}
    pz = {q: (1 + np.cos(tq)) / 2, nz + 1 - q: (np.cos(tq) - 1) / 2}
    lam_c = (2 - 2 * np.cos(2 * tp)) + (2 - 2 * np.cos(2 * tq)) - sym.c[1]
    coarse = s[(p, q)] ** 2 * sym.lam(0, p, q) * rx[p] * rz[q] / lam_c
    # S^2 v, minus the prolonged coarse correction, then S^2 again on each harmonic
    expect = {k: s[k] ** 2 * ((s[(p, q)] ** 2 if k == (p, q) else 0.0) - px[k[0]] * pz[k[1]] * coarse)
              for k in fam}
    Ev_expect = _synth(expect, nx, nz)
    err = np.linalg.norm(Ev - Ev_expect) / np.linalg.norm(Ev_expect)
    assert err <= 1e-12, err


def test_symbol_comparison_separates_v_from_w():
    """The comparison above is sensitive to the recursion: the V- and
    W-cycle symbols on three levels differ by far more than the tolerance."""
    nx, nz = 31, 15
    b = _random_coef(nx, nz, seed=9)
    xs = [_synth(Symbol(nx, nz, 3, 20.0, 2 * np.pi * 5.0, cycle=c).cycle_from_zero(b), nx, nz) for c in (1, 2)]
    assert np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1]) > 1e-4


def test_coarse_stretch_arrays_sample_the_fine_profile():
    """Coarse node I of level l sits on fine node 2I+1 and its half node I-1/2
    on fine node 2I: the layer's stretch factors of level 1 are the fine
    level's values at those nodes (one continuous profile, Collino & Tsogka)."""
    g = FI.Grid(nx=41, nz=23, npml=8, h=20.0, pml_c=3000.0)
    om = 2 * np.pi * 4.0
    f0 = G.stretch_arrays(g, om, 0)
    f1 = G.stretch_arrays(g, om, 1)
    assert f1["h"] == 2 * f0["h"]
    np.testing.assert_allclose(f1["X"], f0["X"][1:2 * f1["nx"]:2], rtol=1e-15)
    np.testing.assert_allclose(f1["Z"], f0["Z"][1:2 * f1["nz"]:2], rtol=1e-15)
    np.testing.assert_allclose(f1["Xh"][:f1["nx"]], f0["X"][0:2 * f1["nx"]:2], rtol=1e-15)
    np.testing.assert_allclose(f1["Zh"][:f1["nz"]], f0["Z"][0:2 * f1["nz"]:2], rtol=1e-15)


def test_level_gamma_preserves_linear_functions_inside():
    """Normalised full weighting reproduces a linear gamma at every coarse node
    whose nine fine neighbours exist (weights (1,2,1)x(1,2,1)/16)."""
    from oracle import helmholtz as H
    g = FI.Grid(nx=41, nz=23, npml=0, h=20.0)
    j, i = np.meshgrid(np.arange(23), np.arange(41), indexing="ij")
    lin = 2.0 + 0.3 * i - 0.7 * j
    c = H.level_gamma(g, lin, 1)
    J, I = np.meshgrid(np.arange(c.shape[0]), np.arange(c.shape[1]), indexing="ij")
    inner = (2 * I + 2 < 41) & (2 * J + 2 < 23)
    np.testing.assert_allclose(c[inner], (2.0 + 0.3 * (2 * I + 1) - 0.7 * (2 * J + 1))[inner], rtol=1e-14, atol=1e-13)
