"""Parity of the CUDA path (through the C ABI) with the oracle, element by
element, on seeded inputs that span several row tiles and ragged batches of
two different grids.  Tolerances: complex128 kernels 1e-10 relative (rounding
order only), complex64 kernels 2e-5 relative (single-precision stencil
arithmetic on O(1) entries), wavefields 1e-5 (the stated target), KKT relative
residual 1e-6 and model update 1e-5 against the direct solve."""
import numpy as np
import pytest

import fwi_inputs as FI
from oracle import fwi, kkt, krylov, mg
from oracle import grid as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _workloads():
    a = FI.tiny_workload(seed=0)
    b = FI.micro_workload(seed=1, nx=37, nz=23, npml=6, n_src=3, n_rec=5, freq=4.0)
    b.survey.freqs_hz = [4.0, 6.5]
    return [a, b]


@pytest.fixture(scope="module")
def setup(lib):
    import paper_2204_06489_gb300 as P
    wls = _workloads()
    f = P.from_workload(wls)
    probs = [fwi.Problem.create(w.grid, w.survey, w.gamma_start) for w in wls]
    d_obs = []
    for i, (w, p) in enumerate(zip(wls, probs)):
        d = fwi.sample(p, fwi.forward(p, w.gamma_true.ravel()))
        d_obs.append(d)
        nf, ns = w.survey.n_freq, w.survey.n_src
        arr = np.zeros((nf, int(w.survey.rec_offsets[-1])), dtype=complex)
        for b in range(p.n_blocks):
            k = p.block_src(b)
            arr[p.block_freq(b), w.survey.rec_offsets[k]:w.survey.rec_offsets[k + 1]] = d[b]
        f.set_observed(i, arr)
    return P, f, wls, probs, d_obs


def _split(wls, probs, field):
    """Field (all blocks) -> list per instance of [B_i, N_i] arrays."""
    out, o = [], 0
    for w, p in zip(wls, probs):
        Nz, Nx = G.padded_shape(w.grid)
        n = p.n_blocks * Nz * Nx
        out.append(field[o:o + n].reshape(p.n_blocks, Nz * Nx))
        o += n
    return out


def _rand_field(n, seed, dtype=torch.complex128):
    g = np.random.default_rng(seed)
    z = g.standard_normal(n) + 1j * g.standard_normal(n)
    return torch.from_numpy(z).to(dtype).cuda(), z


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("prec,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-6)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_helmholtz_operator(setup, prec, tol, adjoint):
    P, f, wls, probs, _ = setup
    lay = f.layout()
    xt, x = _rand_field(lay["field_elems"], 3, prec)
    y = f.apply_helmholtz(xt, adjoint=adjoint).cpu().numpy().astype(np.complex128)
    xs = _split(wls, probs, x if prec == torch.complex128 else xt.cpu().numpy().astype(complex))
    ys = _split(wls, probs, y)
    for i, (w, p) in enumerate(zip(wls, probs)):
        for b in range(p.n_blocks):
            A = p.operator(w.gamma_start.ravel(), p.block_freq(b))
            ref = np.conj(A @ np.conj(xs[i][b])) if adjoint else A @ xs[i][b]
            assert _rel(ys[i][b], ref) < tol, (i, b, _rel(ys[i][b], ref))


def test_adjoint_identity(setup):
    """<A u, v> = <u, A^H v> with the CUDA operator (complex128)."""
    P, f, wls, probs, _ = setup
    n = f.layout()["field_elems"]
    u, _ = _rand_field(n, 4)
    v, _ = _rand_field(n, 5)
    lhs = torch.vdot(v, f.apply_helmholtz(u)).item()
    rhs = torch.vdot(f.apply_helmholtz(v, adjoint=True), u).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _oracle_hier(P, w, p, fidx, opts):
    return mg.Hierarchy(w.grid, p.omegas[fidx], p.gamma_pad(w.gamma_start.ravel()), shift=opts.shift_beta,
                        nu1=opts.nu1, nu2=opts.nu2, wj=opts.omega_jac, cycle=opts.mg_cycle,
                        sigma_cap=opts.sigma_cap, wdepth=opts.mg_wdepth)


@pytest.mark.parametrize("cycle,wdepth", [(1, 2), (2, 2), (2, 9)])
def test_multigrid_cycle(setup, cycle, wdepth):
    _check_cycle(setup, cycle, wdepth, 2, 2)


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (1, 3), (3, 0)])
def test_multigrid_cycle_sweep_counts(setup, nu1, nu2):
    """Odd and uneven sweep counts (single sweeps next to fused pairs, the
    p-update fusion falling back, no post-smoothing)."""
    _check_cycle(setup, 2, 2, nu1, nu2)


def _check_cycle(setup, cycle, wdepth, nu1, nu2):
    P, f, wls, probs, _ = setup
    opts = P.default_opts(mg_cycle=cycle, mg_wdepth=wdepth, nu1=nu1, nu2=nu2)
    n = f.layout()["field_elems"]
    bt, b = _rand_field(n, 6)
    x = f.mg_cycle(bt, opts).cpu().numpy()
    bs, xs = _split(wls, probs, b), _split(wls, probs, x)
    for i, (w, p) in enumerate(zip(wls, probs)):
        hs = {}
        for blk in range(p.n_blocks):
            fi = p.block_freq(blk)
            if fi not in hs:
                hs[fi] = _oracle_hier(P, w, p, fi, opts)
            ref = hs[fi].vcycle(bs[i][blk])
            assert _rel(xs[i][blk], ref) < 1e-10, (i, blk, _rel(xs[i][blk], ref))
    x32 = f.mg_cycle(bt.to(torch.complex64), opts).cpu().numpy().astype(complex)
    assert _rel(x32, x) < 1e-4


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("nu", [2, 1])
def test_inner_solve(setup, adjoint, nu):
    """Batched BiCGStab + multigrid, 6 iterations, complex128, against the
    oracle's same iteration per block (nu = 1: single sweeps, the p update
    outside the smoother)."""
    P, f, wls, probs, _ = setup
    opts = P.default_opts(inner_iters=6, nu1=nu, nu2=nu)
    n = f.layout()["field_elems"]
    bt, b = _rand_field(n, 7)
    x = f.inner_solve(bt, opts, adjoint=adjoint).cpu().numpy()
    bs, xs = _split(wls, probs, b), _split(wls, probs, x)
    for i, (w, p) in enumerate(zip(wls, probs)):
        for blk in range(p.n_blocks):
            fi = p.block_freq(blk)
            h = _oracle_hier(P, w, p, fi, opts)
            A = p.operator(w.gamma_start.ravel(), fi)
            ref, _ = mg.inner_solve(A, h, bs[i][blk], 6, adjoint=adjoint)
            assert _rel(xs[i][blk], ref) < 1e-8, (i, blk, _rel(xs[i][blk], ref))


def test_inner_solve_zero_rhs_block(setup):
    """A block with a zero right-hand side stays exactly zero (no NaN)."""
    P, f, wls, probs, _ = setup
    n = f.layout()["field_elems"]
    bt, _ = _rand_field(n, 8)
    Nz, Nx = G.padded_shape(wls[0].grid)
    bt[:Nz * Nx] = 0
    x = f.inner_solve(bt, P.default_opts(inner_iters=4))
    assert torch.all(x[:Nz * Nx] == 0)
    assert torch.isfinite(torch.view_as_real(x)).all()


@pytest.fixture(scope="module")
def forward_done(setup):
    P, f, wls, probs, d_obs = setup
    d_pred, mis, st = f.forward(P.default_opts())
    return d_pred, mis, st


def test_forward_wavefields_and_misfit(setup, forward_done):
    P, f, wls, probs, d_obs = setup
    d_pred, mis, st = forward_done
    u = f.wavefields().cpu().numpy()
    us = _split(wls, probs, u)
    for i, (w, p) in enumerate(zip(wls, probs)):
        ref = fwi.forward(p, w.gamma_start.ravel())
        for b in range(p.n_blocks):
            assert _rel(us[i][b], ref[b]) < 1e-5, (i, b, _rel(us[i][b], ref[b]))
        r = fwi.residual(p, ref, d_obs[i])
        assert abs(mis[i] - fwi.misfit(p, r)) <= 1e-6 * fwi.misfit(p, r)
        q = fwi.sample(p, ref)
        for b in range(p.n_blocks):
            k = p.block_src(b)
            got = d_pred[i][p.block_freq(b), w.survey.rec_offsets[k]:w.survey.rec_offsets[k + 1]]
            assert _rel(got, q[b]) < 1e-5


def _oracle_kkts(wls, probs, d_obs, eps, include):
    return [kkt.KKT(p, w.gamma_start.ravel(), d, eps, include_Ls_n=include) for w, p, d in zip(wls, probs, d_obs)]


def _pack_gpu(Ks, parts):
    """Per-instance (du, ds, lm) -> GPU packed [du all | lm all | ds all]."""
    du = np.concatenate([p[0].ravel() for p in parts])
    lm = np.concatenate([p[2].ravel() for p in parts])
    ds = np.concatenate([p[1].ravel() for p in parts])
    return np.concatenate([du.view(np.float64), lm.view(np.float64), ds])


def _unpack_gpu(Ks, x):
    nf = sum(K.B * K.N for K in Ks)
    du = x[:2 * nf].view(np.complex128)
    lm = x[2 * nf:4 * nf].view(np.complex128)
    ds = x[4 * nf:]
    out, o, oc = [], 0, 0
    for K in Ks:
        n = K.B * K.N
        out.append((du[o:o + n].reshape(K.B, K.N), ds[oc:oc + K.Nc], lm[o:o + n].reshape(K.B, K.N)))
        o += n
        oc += K.Nc
    return out


@pytest.mark.parametrize("prec,tol", [(torch.float64, 1e-9), (torch.float32, 2e-5)])
def test_kkt_matvec(setup, forward_done, prec, tol):
    P, f, wls, probs, d_obs = setup
    eps = 1e-2
    Ks = _oracle_kkts(wls, probs, d_obs, eps, True)
    rng = np.random.default_rng(9)
    parts = [(rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N)), rng.standard_normal(K.Nc),
              rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N))) for K in Ks]
    x = _pack_gpu(Ks, parts)
    y = f.apply_kkt(torch.from_numpy(x).to(prec).cuda(), P.default_opts(eps=eps)).cpu().numpy().astype(np.float64)
    got = _unpack_gpu(Ks, y)
    for K, p, g in zip(Ks, parts, got):
        ref = K.unpack(K.matvec(K.pack(*p)))
        for a, r in zip(g, ref):
            assert _rel(a, r) < tol, _rel(a, r)


def test_preconditioner_apply(setup, forward_done):
    """One application of the inexact block-triangular preconditioner (eq.
    precond_approx, 4 inner iterations), complex128, against the oracle."""
    P, f, wls, probs, d_obs = setup
    eps = 1e-2
    opts = P.default_opts(eps=eps, inner_iters=4)
    Ks = _oracle_kkts(wls, probs, d_obs, eps, True)
    rng = np.random.default_rng(10)
    parts = [(rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N)), rng.standard_normal(K.Nc),
              rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N))) for K in Ks]
    z = f.apply_precond(torch.from_numpy(_pack_gpu(Ks, parts)).cuda(), opts).cpu().numpy()
    got = _unpack_gpu(Ks, z)
    for i, (K, w, p, pr, g) in enumerate(zip(Ks, wls, probs, parts, got)):
        hs = {fi: _oracle_hier(P, w, p, fi, opts) for fi in range(w.survey.n_freq)}

        def inner(b, rhs, adj):
            fi = p.block_freq(b)
            return mg.inner_solve(K.A[fi], hs[fi], rhs, 4, adj)[0]
        ref = K.unpack(K.precond(K.pack(*pr), inner))
        for a, r in zip(g, ref):
            assert _rel(a, r) < 1e-8, _rel(a, r)


@pytest.fixture(scope="module")
def direct_updates(setup):
    """The oracle's model update per instance from the sparse direct solve of
    the whole KKT system (eps = 1e-2, with the -L s_n term)."""
    P, f, wls, probs, d_obs = setup
    return [K.delta_s(K.solve_direct()) for K in _oracle_kkts(wls, probs, d_obs, 1e-2, True)]


@pytest.mark.parametrize("prec", [0, 1])
def test_kkt_solve_matches_direct(setup, forward_done, direct_updates, prec):
    """Whole KKT solve (both instances jointly) against the oracle's sparse
    direct solve per instance: relative residual <= 1e-6 recomputed in FP64 and
    model update within 1e-5."""
    P, f, wls, probs, d_obs = setup
    eps = 1e-2
    opts = P.default_opts(eps=eps, precision=prec, tol=1e-7, inner_iters=6)
    ds, st = f.kkt_solve(opts)
    assert st["rel_res"] <= 1e-7
    o = 0
    for ref in direct_updates:
        got = ds[o:o + ref.size]
        o += ref.size
        assert _rel(got, ref) < 1e-5, _rel(got, ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_kkt_solve_with_outer_bicgstab(setup, forward_done, direct_updates, prec):
    """The memory-lean outer solver (BiCGStab in the real inner product, the
    option of Sec. 7) reaches the same, unique KKT update as the oracle's
    direct solve, with the FP64 residual <= 1e-7."""
    P, f, wls, probs, d_obs = setup
    eps = 1e-2
    opts = P.default_opts(eps=eps, precision=prec, tol=1e-7, inner_iters=6, outer_solver=1)
    ds, st = f.kkt_solve(opts)
    assert st["rel_res"] <= 1e-7
    o = 0
    for ref in direct_updates:
        got = ds[o:o + ref.size]
        o += ref.size
        assert _rel(got, ref) < 1e-5, _rel(got, ref)


def test_gradient_matches_oracle(setup):
    P, f, wls, probs, d_obs = setup
    mis, g, st = f.gradient(P.default_opts())
    o = 0
    for w, p, d, m in zip(wls, probs, d_obs, mis):
        phi, gr = fwi.gradient(p, w.gamma_start.ravel(), d)
        n = gr.size
        assert _rel(g[o:o + n], gr) < 1e-4, _rel(g[o:o + n], gr)
        assert abs(m - phi) <= 1e-6 * phi
        o += n


def test_invalid_calls_return_errors(setup):
    P, f, wls, probs, d_obs = setup
    bad = P.default_opts(restart=0)
    with pytest.raises(P.FwiError) as e:
        f.kkt_solve(bad)
    assert e.value.code == P.FWI_E_INVAL
    with pytest.raises(P.FwiError) as e:
        f.set_model(0, -np.ones((wls[0].grid.nz, wls[0].grid.nx)))
    assert e.value.code == P.FWI_E_NUMERIC


def test_kkt_solve_odd_control_size(lib):
    """A control vector of odd length (15 x 11 core) makes the packed KKT
    length odd; the Krylov basis must still be aligned for complex loads."""
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=3, nx=15, nz=11, npml=4, n_src=2, n_rec=3)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    obs = np.zeros((1, int(wl.survey.rec_offsets[-1])), dtype=complex)
    for b in range(prob.n_blocks):
        k = prob.block_src(b)
        obs[0, wl.survey.rec_offsets[k]:wl.survey.rec_offsets[k + 1]] = d[b]
    f = P.from_workload(wl)
    f.set_observed(0, obs)
    assert f.layout()["kkt_elems"] % 2 == 1
    opts = P.default_opts(eps=1e-2, tol=1e-7)
    f.forward(opts)
    ds, st = f.kkt_solve(opts)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    ref = K.delta_s(K.solve_direct())
    assert st["rel_res"] <= 1e-7 and _rel(ds, ref) < 1e-5
    f.close()


@pytest.mark.parametrize("prec,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-6)])
def test_wide_grid_operator_and_cycle(lib, prec, tol):
    """A wide grid (313 padded columns: ten 30-column strips and a ragged 13 for
    the operator, five 60-column strips and a ragged 13 for the smoother) taller
    than one strip band; operator, adjoint and one multigrid cycle against the
    oracle."""
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=11, nx=301, nz=29, npml=6, n_src=2, n_rec=7, freq=6.0)
    f = P.from_workload(wl)
    p = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    n = f.layout()["field_elems"]
    xt, x = _rand_field(n, 12, prec)
    xs = x if prec == torch.complex128 else xt.cpu().numpy().astype(complex)
    A = p.operator(wl.gamma_start.ravel(), 0)
    N = A.shape[0]
    for adj in (False, True):
        y = f.apply_helmholtz(xt, adjoint=adj).cpu().numpy().astype(complex)
        for b in range(p.n_blocks):
            xb = xs[b * N:(b + 1) * N]
            ref = np.conj(A @ np.conj(xb)) if adj else A @ xb
            assert _rel(y[b * N:(b + 1) * N], ref) < tol
    opts = P.default_opts()
    xc = f.mg_cycle(xt, opts).cpu().numpy().astype(complex)
    h = _oracle_hier(P, wl, p, 0, opts)
    for b in range(p.n_blocks):
        ref = h.vcycle(xs[b * N:(b + 1) * N])
        assert _rel(xc[b * N:(b + 1) * N], ref) < (1e-10 if prec == torch.complex128 else 2e-4)
    f.close()


def test_exact_block_mode_is_gmres_full(lib):
    """The paper's GMRes-full on the GPU: with the block solves run to 1e-12
    (inner_tol, complex128) the preconditioner is the exact one of Sec. 5, so
    FGMRES ends within rank(F) + 1 iterations (micro grid, 2 sources x 3
    receivers: rank(F) = 12) and its update matches the direct KKT solve."""
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=0)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    obs = np.zeros((1, int(wl.survey.rec_offsets[-1])), dtype=complex)
    for b in range(prob.n_blocks):
        k = prob.block_src(b)
        obs[0, wl.survey.rec_offsets[k]:wl.survey.rec_offsets[k + 1]] = d[b]
    f = P.from_workload(wl)
    f.set_observed(0, obs)
    opts = P.default_opts(eps=1e-2, tol=1e-10, precision=0, inner_tol=1e-12, restart=40, fwd_tol=1e-12)
    f.forward(opts)
    ds, st = f.kkt_solve(opts)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    rankF = 2 * int(np.count_nonzero(K.Fd))
    assert rankF == 12
    assert st["outer_iters"] <= rankF + 1, st["outer_iters"]
    assert st["rel_res"] <= 1e-10
    assert _rel(ds, K.delta_s(K.solve_direct())) < 1e-8
    f.close()


@pytest.mark.parametrize("adjoint", [False, True])
def test_inner_solve_with_ilu0(setup, adjoint):
    """BiCGStab preconditioned by ILU(0) of A' (the incomplete-LU block
    approximation of Sec. 5 with zero fill; wavefront substitutions on the
    GPU), complex128, 5 iterations, against the oracle's same iteration."""
    from oracle.ilu import ILU0
    P, f, wls, probs, _ = setup
    opts = P.default_opts(inner_iters=5, inner_solver=1)
    n = f.layout()["field_elems"]
    bt, b = _rand_field(n, 17)
    x = f.inner_solve(bt, opts, adjoint=adjoint).cpu().numpy()
    bs, xs = _split(wls, probs, b), _split(wls, probs, x)
    for i, (w, p) in enumerate(zip(wls, probs)):
        Nz, Nx = G.padded_shape(w.grid)
        for blk in range(p.n_blocks):
            A = p.operator(w.gamma_start.ravel(), p.block_freq(blk))
            F = ILU0(A, Nz, Nx)
            if adjoint:
                ref = np.conj(krylov.bicgstab(lambda v: A @ v, np.conj(bs[i][blk]), F.solve, iters=5, tol=0.0)[0])
            else:
                ref = krylov.bicgstab(lambda v: A @ v, bs[i][blk], F.solve, iters=5, tol=0.0)[0]
            assert _rel(xs[i][blk], ref) < 1e-8, (i, blk, _rel(xs[i][blk], ref))


def test_preconditioner_with_ilu0_blocks(setup, forward_done):
    """The paper's inexact preconditioner with A~ = ILU(0) (inner_solver 2: one
    factorised application per block, no Krylov iteration), complex128,
    against the oracle's eq. precond_approx with the same A~."""
    from oracle.ilu import ILU0
    P, f, wls, probs, d_obs = setup
    eps = 1e-2
    opts = P.default_opts(eps=eps, inner_solver=2)
    Ks = _oracle_kkts(wls, probs, d_obs, eps, True)
    rng = np.random.default_rng(18)
    parts = [(rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N)), rng.standard_normal(K.Nc),
              rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N))) for K in Ks]
    z = f.apply_precond(torch.from_numpy(_pack_gpu(Ks, parts)).cuda(), opts).cpu().numpy()
    got = _unpack_gpu(Ks, z)
    for K, w, p, pr, g in zip(Ks, wls, probs, parts, got):
        Nz, Nx = G.padded_shape(w.grid)
        Fs = {fi: ILU0(K.A[fi], Nz, Nx) for fi in range(w.survey.n_freq)}

        def inner(b, rhs, adj):
            F = Fs[p.block_freq(b)]
            return F.solve_adjoint(rhs) if adj else F.solve(rhs)
        ref = K.unpack(K.precond(K.pack(*pr), inner))
        for a, r in zip(g, ref):
            assert _rel(a, r) < 1e-9, _rel(a, r)
