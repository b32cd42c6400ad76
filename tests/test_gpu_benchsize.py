"""Parity with the oracle on the benchmark's own grid: the 401x141 Marmousi-
shaped model with its 20-node layer (441x181 padded, six multigrid levels;
complex64 runs levels 0-1 in global memory and 2-5 in the shared-memory
kernel, from 110x45 down), two sources x 3 and 7 Hz = 4 blocks, in the launch
configuration the benchmark uses (same kernels, tables and cycle).
Tolerances as in test_gpu_parity: complex128 kernels 1e-10 (multigrid) and
1e-8 (BiCGStab), complex64 cycle within 1e-4 of complex128, wavefields 1e-5,
gradient 1e-4, KKT model update 1e-5 at relative residual <= 1e-7."""
import numpy as np
import pytest

import fwi_inputs as FI
from oracle import fwi, kkt, krylov, mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = 0.1


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture(scope="module")
def bench(lib):
    import paper_2204_06489_gb300 as P
    wl = FI.marmousi_shaped_workload(n_src=2, freqs=(3.0, 7.0))
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    f = P.from_workload(wl)
    obs = np.zeros((wl.survey.n_freq, int(wl.survey.rec_offsets[-1])), dtype=complex)
    for b in range(prob.n_blocks):
        k = prob.block_src(b)
        obs[prob.block_freq(b), wl.survey.rec_offsets[k]:wl.survey.rec_offsets[k + 1]] = d[b]
    f.set_observed(0, obs)
    yield P, f, wl, prob, d
    f.close()


def _hier(P, wl, prob, fi, opts):
    return mg.Hierarchy(wl.grid, prob.omegas[fi], prob.gamma_pad(wl.gamma_start.ravel()), shift=opts.shift_beta,
                        nu1=opts.nu1, nu2=opts.nu2, wj=opts.omega_jac, cycle=opts.mg_cycle,
                        sigma_cap=opts.sigma_cap, wdepth=opts.mg_wdepth)


def _field(n, seed):
    g = np.random.default_rng(seed)
    z = g.standard_normal(n) + 1j * g.standard_normal(n)
    return torch.from_numpy(z).cuda(), z


def test_levels_of_the_benchmark_grid(bench):
    P, f, wl, prob, d = bench
    h = _hier(P, wl, prob, 0, P.default_opts())
    assert h.levels == 6 and h.shapes[2] == (45, 110) and h.shapes[-1] == (5, 13)


@pytest.mark.parametrize("cycle,wdepth", [(2, 2), (1, 2), (2, 1)])
def test_multigrid_cycle_at_benchmark_size(bench, cycle, wdepth):
    P, f, wl, prob, d = bench
    opts = P.default_opts(mg_cycle=cycle, mg_wdepth=wdepth)
    N = prob.operator(wl.gamma_start.ravel(), 0).shape[0]
    bt, b = _field(prob.n_blocks * N, 31)
    x = f.mg_cycle(bt, opts).cpu().numpy()
    hs = {fi: _hier(P, wl, prob, fi, opts) for fi in range(wl.survey.n_freq)}
    for blk in range(prob.n_blocks):
        ref = hs[prob.block_freq(blk)].vcycle(b[blk * N:(blk + 1) * N])
        assert _rel(x[blk * N:(blk + 1) * N], ref) < 1e-10, (blk, _rel(x[blk * N:(blk + 1) * N], ref))
    x32 = f.mg_cycle(bt.to(torch.complex64), opts).cpu().numpy().astype(complex)
    for blk in range(prob.n_blocks):
        sl = slice(blk * N, (blk + 1) * N)
        assert _rel(x32[sl], x[sl]) < 1e-4, (blk, _rel(x32[sl], x[sl]))


@pytest.mark.parametrize("adjoint", [False, True])
def test_inner_solve_at_benchmark_size(bench, adjoint):
    P, f, wl, prob, d = bench
    opts = P.default_opts(inner_iters=6)
    N = prob.operator(wl.gamma_start.ravel(), 0).shape[0]
    bt, b = _field(prob.n_blocks * N, 32)
    x = f.inner_solve(bt, opts, adjoint=adjoint).cpu().numpy()
    for blk in range(prob.n_blocks):
        fi = prob.block_freq(blk)
        A = prob.operator(wl.gamma_start.ravel(), fi)
        ref, _ = mg.inner_solve(A, _hier(P, wl, prob, fi, opts), b[blk * N:(blk + 1) * N], 6, adjoint=adjoint)
        assert _rel(x[blk * N:(blk + 1) * N], ref) < 1e-8, (blk, _rel(x[blk * N:(blk + 1) * N], ref))


@pytest.fixture(scope="module")
def forward_bench(bench):
    P, f, wl, prob, d = bench
    return f.forward(P.default_opts(eps=EPS))


def test_forward_at_benchmark_size(bench, forward_bench):
    """complex64 inner solves with FP64 refinement (the benchmark's forward
    modelling) against the sparse LU wavefields."""
    P, f, wl, prob, d = bench
    d_pred, mis, st = forward_bench
    u = f.wavefields().cpu().numpy()
    ref = fwi.forward(prob, wl.gamma_start.ravel())
    N = ref.shape[1]
    for blk in range(prob.n_blocks):
        assert _rel(u[blk * N:(blk + 1) * N], ref[blk]) < 1e-5, blk
    phi = fwi.misfit(prob, fwi.residual(prob, ref, d))
    assert abs(mis[0] - phi) <= 1e-6 * phi


@pytest.fixture(scope="module")
def oracle_gmres_full(bench):
    """The paper's GMRes-full: GMRES(30) with the exact block-triangular
    preconditioner (LU block solves), to 1e-10."""
    P, f, wl, prob, d = bench
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, EPS, include_Ls_n=True)
    x, info = krylov.fgmres(K.matvec, K.rhs(), K.precond, restart=30, tol=1e-10, max_iter=300)
    assert info["true_relres"] <= 1e-10
    return K, K.delta_s(x), info


@pytest.mark.parametrize("prec", [1, 0])
def test_kkt_solve_at_benchmark_size(bench, forward_bench, oracle_gmres_full, prec):
    """The benchmark's KKT solve (inexact preconditioner, complex64 bulk with
    FP64 refinement; or complex128) against the oracle's exact-preconditioner
    GMRES: FP64 residual <= 1e-7 and model update within 1e-5."""
    P, f, wl, prob, d = bench
    K, ds_ref, info = oracle_gmres_full
    opts = P.default_opts(eps=EPS, precision=prec, tol=1e-7, inner_iters=8, check_orth=1)
    ds, st = f.kkt_solve(opts)
    assert st["rel_res"] <= 1e-7
    assert _rel(ds, ds_ref) < 1e-5, _rel(ds, ds_ref)
    # the Arnoldi inner products keep the basis orthogonal to rounding level
    assert st["orth_loss"] < 1e-5, st["orth_loss"]


def test_gradient_at_benchmark_size(bench, forward_bench):
    P, f, wl, prob, d = bench
    mis, g, st = f.gradient(P.default_opts())
    phi, gr = fwi.gradient(prob, wl.gamma_start.ravel(), d)
    assert _rel(g, gr) < 1e-4, _rel(g, gr)
    assert abs(mis[0] - phi) <= 1e-6 * phi


@pytest.mark.parametrize("strip_rows,coarse_threads", [(8, 1024), (32, 512), (5, 1024)])
def test_layout_options_keep_the_cycle(bench, strip_rows, coarse_threads):
    """The autotuned launch layout (column-strip height, threads of the
    shared-memory coarse cycle) changes no arithmetic: complex128 cycle and
    inner solve equal the oracle as with the defaults."""
    P, f, wl, prob, d = bench
    opts = P.default_opts(strip_rows=strip_rows, coarse_threads=coarse_threads, inner_iters=3)
    N = prob.operator(wl.gamma_start.ravel(), 0).shape[0]
    bt, b = _field(prob.n_blocks * N, 33)
    x = f.mg_cycle(bt, opts).cpu().numpy()
    xi = f.inner_solve(bt, opts).cpu().numpy()
    for blk in range(prob.n_blocks):
        fi = prob.block_freq(blk)
        h = _hier(P, wl, prob, fi, opts)
        sl = slice(blk * N, (blk + 1) * N)
        assert _rel(x[sl], h.vcycle(b[sl])) < 1e-10
        ref, _ = mg.inner_solve(prob.operator(wl.gamma_start.ravel(), fi), h, b[sl], 3)
        assert _rel(xi[sl], ref) < 1e-8
