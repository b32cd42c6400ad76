"""GPU checks of the drivers around the KKT solve: the autograd function
(hand-written adjoint), Newton steps (step-wise parity with the oracle),
frequency continuation, batching of independent instances, graph replay and
the two precision forms."""
import numpy as np
import pytest
from scipy.ndimage import gaussian_filter

import fwi_inputs as FI
from oracle import fwi, kkt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _obs_array(wl, prob, d):
    arr = np.zeros((wl.survey.n_freq, int(wl.survey.rec_offsets[-1])), dtype=complex)
    for b in range(prob.n_blocks):
        k = prob.block_src(b)
        arr[prob.block_freq(b), wl.survey.rec_offsets[k]:wl.survey.rec_offsets[k + 1]] = d[b]
    return arr


def _setup(wl):
    import paper_2204_06489_gb300 as P
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
    f = P.from_workload(wl)
    f.set_observed(0, _obs_array(wl, prob, d))
    return P, f, prob, d


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("mode", ["save", "recompute"])
def test_autograd_misfit_gradient(lib, mode):
    """HelmholtzMisfit: backward vs the oracle gradient (<= 1e-4) and vs central
    differences of its own forward along smooth random directions (<= 1e-3;
    16 directions for the recompute strategy, 3 for save)."""
    from paper_2204_06489_gb300.autograd import misfit
    wl = FI.micro_workload(seed=4, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    P, f, prob, d = _setup(wl)
    g0 = torch.tensor(wl.gamma_start, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = misfit(g0, f, mode=mode)
    phi.backward()
    grad = g0.grad.detach().cpu().numpy().ravel()
    phi_o, grad_o = fwi.gradient(prob, wl.gamma_start.ravel(), d)
    assert abs(phi.item() - phi_o) <= 1e-6 * phi_o
    assert _rel(grad, grad_o) < 1e-4
    s0 = wl.gamma_start
    for seed in range(16 if mode == "recompute" else 3):   # 16 smooth directions, seeds 0-15
        dirn = gaussian_filter(np.random.default_rng(seed).standard_normal(s0.shape), 3.0)
        dirn *= 0.003 * s0.mean() / np.abs(dirn).max()
        with torch.no_grad():
            fp = misfit(torch.tensor(s0 + dirn, device="cuda"), f, mode=mode).item()
            fm = misfit(torch.tensor(s0 - dirn, device="cuda"), f, mode=mode).item()
        fd = (fp - fm) / 2
        an = float(np.dot(grad, dirn.ravel()))
        assert abs(fd - an) <= 1e-3 * abs(an), (seed, fd, an)
    f.close()


def test_autograd_save_equals_recompute(lib):
    from paper_2204_06489_gb300.autograd import misfit
    wl = FI.micro_workload(seed=5, nx=31, nz=17, npml=6, n_src=2, n_rec=6)
    P, f, prob, d = _setup(wl)
    gs = []
    for mode in ("save", "recompute"):
        g0 = torch.tensor(wl.gamma_start, dtype=torch.float64, device="cuda", requires_grad=True)
        misfit(g0, f, mode=mode).backward()
        gs.append(g0.grad.cpu().numpy())
    assert _rel(gs[0], gs[1]) < 1e-7
    f.close()


def test_newton_steps_stepwise_parity(lib):
    """Two Gauss-Newton steps on the GPU; at every model s_n the GPU reached,
    the oracle's direct KKT solve gives the same update (<= 1e-5), and the first
    full step lowers the misfit (the trajectory itself is not pinned end to end;
    full steps without line search need not decrease the misfit every time)."""
    wl = FI.micro_workload(seed=6, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    P, f, prob, d = _setup(wl)
    opts = P.default_opts(eps=1e-2, tol=1e-8, include_Ls_n=0)
    mis = []
    for step in range(2):
        s_n = f.get_model(0).ravel()
        _, m, _ = f.forward(opts, want_data=False)
        mis.append(m[0])
        ds, st = f.newton_step(opts)
        K = kkt.KKT(prob, s_n, d, 1e-2, include_Ls_n=False)
        ref = K.delta_s(K.solve_direct())
        assert st["rel_res"] <= 1e-8
        assert _rel(ds, ref) < 1e-5, (step, _rel(ds, ref))
    assert mis[1] < mis[0]
    f.close()


def test_frequency_continuation_reduces_misfit(lib):
    import paper_2204_06489_gb300 as P
    from paper_2204_06489_gb300.newton import frequency_continuation
    wl = FI.micro_workload(seed=7, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    freqs = [3.0, 5.0, 7.0]

    def observed(fq):
        sv = FI.Survey(**{**wl.survey.__dict__, "freqs_hz": [fq]})
        p = fwi.Problem.create(wl.grid, sv, wl.gamma_start)
        dd = fwi.sample(p, fwi.forward(p, wl.gamma_true.ravel()))
        return _obs_array(FI.Workload("x", wl.grid, sv, wl.gamma_true, wl.gamma_start), p, dd)

    opts = P.default_opts(eps=1e-2, include_Ls_n=0)
    g, log = frequency_continuation(wl.grid, wl.survey, wl.gamma_start, observed, freqs, 1, opts)
    assert len(log) == 3
    for st in log:
        assert st["misfit_after"] < st["misfit_before"] if "misfit_after" in st else True
    err0 = np.linalg.norm(wl.gamma_start - wl.gamma_true)
    err1 = np.linalg.norm(g - wl.gamma_true)
    assert err1 < err0


def test_batched_instances_equal_separate_solves(lib):
    """Two instances of different grid sizes solved in one batch give the same
    updates as each solved alone (independent problems; ragged launches)."""
    import paper_2204_06489_gb300 as P
    wa = FI.micro_workload(seed=8, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    wb = FI.micro_workload(seed=9, nx=29, nz=25, npml=6, n_src=2, n_rec=5, freq=6.0)
    opts = P.default_opts(eps=1e-2, tol=1e-8)
    sep = []
    datas = []
    for w in (wa, wb):
        Pm, f, prob, d = _setup(w)
        datas.append(_obs_array(w, prob, d))
        f.forward(opts, want_data=False)
        ds, st = f.kkt_solve(opts)
        sep.append(ds)
        f.close()
    fb = P.from_workload([wa, wb])
    fb.set_observed(0, datas[0])
    fb.set_observed(1, datas[1])
    fb.forward(opts, want_data=False)
    ds, st = fb.kkt_solve(opts)
    n0 = wa.grid.nx * wa.grid.nz
    assert _rel(ds[:n0], sep[0]) < 1e-6
    assert _rel(ds[n0:], sep[1]) < 1e-6
    fb.close()


def test_graph_replay_equals_direct_launches_and_precisions_agree(lib):
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=10, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    Pm, f, prob, d = _setup(wl)
    out = {}
    for name, kw in (("graph", dict(use_graph=1)), ("direct", dict(use_graph=0)),
                     ("c128", dict(precision=P.FWI_C128))):
        opts = P.default_opts(eps=1e-2, tol=1e-8, **kw)
        f.forward(opts, want_data=False)
        ds, st = f.kkt_solve(opts)
        assert st["rel_res"] <= 1e-8
        out[name] = ds
        out[name + "_iters"] = st["outer_iters"]
    assert _rel(out["graph"], out["direct"]) < 1e-12
    assert out["graph_iters"] == out["direct_iters"]
    assert _rel(out["c128"], out["graph"]) < 1e-6
    f.close()


@pytest.mark.parametrize("restart,max_outer", [(5, 600), (4, 9)])
def test_device_controlled_cycles_equal_the_host_loop(lib, restart, max_outer):
    """With graph replay the FGMRES restart cycle runs as one CUDA graph under
    device control (a WHILE node over the Arnoldi steps, the step index and
    the convergence test on the device).  Over several restarts, and when the
    iteration cap stops the solve (FWI_E_NOCONV), it takes the same steps as
    the host-driven loop: same iteration count, same update."""
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=12, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    Pm, f, prob, d = _setup(wl)
    res = {}
    for g in (1, 0):
        opts = P.default_opts(eps=1e-2, tol=1e-8, restart=restart, max_outer=max_outer, use_graph=g)
        f.forward(opts, want_data=False)
        ds, st = f.kkt_solve(opts, allow_noconv=True)
        res[g] = (ds, st)
    assert res[1][1]["outer_iters"] == res[0][1]["outer_iters"]
    assert res[1][1]["refinements"] == res[0][1]["refinements"]
    assert _rel(res[1][0], res[0][0]) < 1e-12
    if max_outer < 100:
        assert res[1][1]["outer_iters"] == max_outer and res[1][1]["rel_res"] > 1e-8
    else:
        assert res[1][1]["rel_res"] <= 1e-8
    f.close()


def test_autotuner_picks_a_converging_schedule(lib):
    import paper_2204_06489_gb300 as P
    from paper_2204_06489_gb300.autotune import tune_inner
    wl = FI.tiny_workload()
    f = P.from_workload(wl)
    n = f.layout()["field_elems"]
    g = np.random.default_rng(1)
    b = torch.from_numpy((g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)).cuda()
    best, table = tune_inner(f, b, P.default_opts(inner_iters=3), nus=(1, 2), omegas=(0.5,), wdepths=(1, 2))
    assert len(table) == 4
    rates = {(t[0], t[2]): t[6] for t in table}
    assert rates[(best.nu1, best.mg_wdepth)] == max(rates.values())
    assert all(t[4] < 1.0 for t in table)
    f.close()


def test_single_level_grid_kkt_solve(lib):
    """A padded grid of at most 256 nodes has one multigrid level: the whole
    cycle is the shared-memory kernel's exact coarsest solve, and the level-0
    strip kernels (operator apply with the BiCGStab dots) still run.  The KKT
    solution must match the oracle's direct solve."""
    wl = FI.micro_workload(seed=11, nx=7, nz=5, npml=4, n_src=2, n_rec=3)
    assert (wl.grid.nx + 2 * wl.grid.npml) * (wl.grid.nz + 2 * wl.grid.npml) <= 256
    P, f, prob, d = _setup(wl)
    opts = P.default_opts(eps=1e-2, tol=1e-7)
    f.forward(opts)
    ds, st = f.kkt_solve(opts)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    ref = K.delta_s(K.solve_direct())
    assert st["rel_res"] <= 1e-7
    assert _rel(ds, ref) < 1e-5
    f.close()


def test_reduced_space_cg_step_equals_the_kkt_solution(lib):
    """RSGN-CG (the paper's reduced-space comparison method): the normal
    equations by CG give the same unique update as the KKT system; checked
    against the oracle's direct KKT solve and against the library's own
    full-space step from the same model."""
    wl = FI.micro_workload(seed=12, nx=31, nz=17, npml=6, n_src=2, n_rec=6)
    P, f, prob, d = _setup(wl)
    opts = P.default_opts(eps=1e-2, tol=1e-9, max_outer=400)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    ref = K.delta_s(K.solve_direct())
    ds_cg, st = f.rsgn_step(opts)
    assert st["outer_iters"] > 1 and st["rel_res"] <= 1e-9
    assert _rel(ds_cg, ref) < 1e-6, _rel(ds_cg, ref)
    f.set_model(0, wl.gamma_start)
    ds_kkt, _ = f.newton_step(P.default_opts(eps=1e-2, tol=1e-7))
    assert _rel(ds_cg, ds_kkt) < 1e-5
    f.close()


def test_gauss_newton_lambda_max_matches_oracle(lib):
    """fwi_normal_lambda_max (power iteration on the matrix-free normal
    operator, the regulariser rule eps = alpha * lambda_max) against the
    oracle's same iteration from the same start vector, and below the dense
    largest eigenvalue."""
    wl = FI.micro_workload(seed=6, nx=31, nz=17, npml=6, n_src=3, n_rec=6)
    wl.survey.rec_w = np.random.default_rng(3).uniform(0.5, 2.0, wl.survey.rec_w.shape)
    P, f, prob, d = _setup(wl)
    opts = P.default_opts(eps=1e-2, fwd_tol=1e-11)
    f.forward(opts)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    ref = K.gn_lambda_max(6)
    lam, st = f.normal_lambda_max(opts, iters=6)
    assert abs(lam - ref[-1]) <= 1e-6 * ref[-1], (lam, ref[-1])
    Hm, _ = K.normal_system()
    assert lam <= np.linalg.eigvalsh(Hm - K.eps * np.eye(K.Nc)).max() * (1 + 1e-9)
    f.close()


@pytest.mark.parametrize("fp64", [2, 1, 0])
def test_arnoldi_dot_precision_options(lib, fp64):
    """The three Arnoldi inner-product forms (compensated Dot2; FP64 products;
    FP32 runs summed in FP64) reach the same KKT update, and the measured loss
    of orthogonality of the complex64 basis stays at single-precision rounding
    level."""
    wl = FI.micro_workload(seed=7, nx=41, nz=21, npml=8, n_src=3, n_rec=8)
    P, f, prob, d = _setup(wl)
    opts = P.default_opts(eps=1e-2, tol=1e-7, arnoldi_dots=fp64, check_orth=1)
    f.forward(opts)
    ds, st = f.kkt_solve(opts)
    K = kkt.KKT(prob, wl.gamma_start.ravel(), d, 1e-2, include_Ls_n=True)
    assert st["rel_res"] <= 1e-7
    assert _rel(ds, K.delta_s(K.solve_direct())) < 1e-5
    assert 0.0 < st["orth_loss"] < 1e-5, st["orth_loss"]
    f.close()


def test_kernel_profile_counts_every_direct_launch(lib):
    """fwi_kernel_profile brackets every direct launch: over one multigrid
    cycle its launch total equals the library's launch counter, and the
    level-0 two-sweep smoother rows carry the stated bytes (five complex
    elements per node from zero, six otherwise)."""
    wl = FI.micro_workload(seed=8, nx=61, nz=31, npml=8, n_src=2, n_rec=5)
    P, f, prob, d = _setup(wl)
    opts = P.default_opts()
    n = f.layout()["field_elems"]
    b = torch.ones(n, dtype=torch.complex64, device="cuda")
    f.mg_cycle(b, opts)                                   # builds the hierarchy
    f.kernel_profile(1)
    l0 = lib.fwi_kernel_launches()
    f.mg_cycle(b, opts)
    launched = lib.fwi_kernel_launches() - l0
    prof = f.kernel_profile(0)
    assert sum(r["launches"] for r in prof["rows"]) == launched
    rows = [r for r in prof["rows"] if r["kernel"] == "k_jacobi2_march" and r["level"] == 0]
    assert len(rows) == 1 and rows[0]["launches"] == 2 and rows[0]["ms"] > 0
    assert rows[0]["bytes"] == (5 + 6) * 8 * n
    assert prof["gaps"] == launched - 1
    f.close()


def test_warm_started_forward_matches_lu(lib):
    """After a small model change the forward solve starts from the previous
    wavefields (fwd_warm) and reaches the same tolerance: wavefields equal the
    oracle's LU solution at the new model within 1e-5, in no more refinement
    sweeps than a cold start."""
    import paper_2204_06489_gb300 as P
    wl = FI.micro_workload(seed=13, nx=61, nz=31, npml=8, n_src=3, n_rec=8)
    Pm, f, prob, d = _setup(wl)
    f.forward(P.default_opts(), want_data=False)
    s1 = wl.gamma_start * (1.0 + 0.01 * gaussian_filter(np.random.default_rng(4).standard_normal(wl.gamma_start.shape), 3.0))
    f.set_model(0, s1)
    _, _, st_w = f.forward(P.default_opts(), want_data=False)
    u_w = f.wavefields().cpu().numpy()
    f.set_model(0, s1)
    _, _, st_c = f.forward(P.default_opts(fwd_warm=0), want_data=False)
    assert st_w["fwd_warm"] == 1 and st_c["fwd_warm"] == 0
    assert st_w["fwd_sweeps"] <= st_c["fwd_sweeps"]
    ref = fwi.forward(prob, s1.ravel())
    N = ref.shape[1]
    for b in range(prob.n_blocks):
        assert _rel(u_w[b * N:(b + 1) * N], ref[b]) < 1e-5
    f.close()


def test_autograd_at_the_differentiation_workload_size(lib):
    """The differentiation workload's size (801 x 281 at h = 10 m, 30-node
    layer, 861 x 341 padded; 64 sources, 801 receivers, 6 Hz; complex64
    wavefields with FP64 refinement, recomputed for the backward pass): the
    hand-written adjoint gradient against central differences of the misfit
    along 16 smooth random directions (Gaussian-filtered noise, 10 cells,
    seeds 0-15), relative error <= 1e-3."""
    import paper_2204_06489_gb300 as P
    from paper_2204_06489_gb300.autograd import misfit
    wl = FI.autograd_workload()
    f = P.FWI([wl.grid])
    f.set_survey(0, wl.survey)
    f.set_model(0, wl.gamma_true)
    d, _, _ = f.forward(P.default_opts(), want_data=True)
    f.set_observed(0, d[0])
    f.set_model(0, wl.gamma_start)
    opts = P.default_opts()
    g0 = torch.tensor(wl.gamma_start, dtype=torch.float64, device="cuda", requires_grad=True)
    phi = misfit(g0, f, mode="recompute", opts=opts)
    phi.backward()
    grad = g0.grad.detach().cpu().numpy()
    s0 = wl.gamma_start
    for seed in range(16):
        dirn = gaussian_filter(np.random.default_rng(seed).standard_normal(s0.shape), 10.0)
        dirn *= 0.003 * s0.mean() / np.abs(dirn).max()
        with torch.no_grad():
            fp = misfit(torch.tensor(s0 + dirn, device="cuda"), f, opts=opts).item()
            fm = misfit(torch.tensor(s0 - dirn, device="cuda"), f, opts=opts).item()
        an = float(np.sum(grad * dirn))
        assert abs((fp - fm) / 2 - an) <= 1e-3 * abs(an), (seed, (fp - fm) / 2, an)
    f.close()
