"""The quasi-Newton H block of the preconditioner (Sec. 5 after eq. precond:
H ~ L may be replaced by L-BFGS; Sec. 7) and the Hessian-vector product
against the oracle, on the two-instance parity problem (tiny 101x51 grid and
a 37x23 grid with two frequencies).

The library applies the L-BFGS inverse in the compact form of Byrd, Nocedal &
Schnabel; the oracle uses the two-loop recursion (oracle/lbfgs.py, pinned by
quadratic termination and the spectral closed form).  Pairs live on the
concatenated control of all instances; pairs supported on one instance give
that instance's own L-BFGS, which is what the oracle computes per instance.
Tolerances: preconditioner 1e-8 (as the eps I preconditioner test), Hessian
product 1e-6 (refined block solves to 1e-9), KKT model update 1e-5 at FP64
residual <= 1e-7."""
import numpy as np
import pytest

import fwi_inputs as FI
from oracle import fwi, kkt, lbfgs, mg
from oracle import grid as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = 1e-2


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture(scope="module")
def setup(lib):
    import paper_2204_06489_gb300 as P
    a = FI.tiny_workload(seed=0)
    b = FI.micro_workload(seed=1, nx=37, nz=23, npml=6, n_src=3, n_rec=5, freq=4.0)
    b.survey.freqs_hz = [4.0, 6.5]
    wls = [a, b]
    f = P.from_workload(wls)
    probs = [fwi.Problem.create(w.grid, w.survey, w.gamma_start) for w in wls]
    d_obs = []
    for i, (w, p) in enumerate(zip(wls, probs)):
        d = fwi.sample(p, fwi.forward(p, w.gamma_true.ravel()))
        d_obs.append(d)
        arr = np.zeros((w.survey.n_freq, int(w.survey.rec_offsets[-1])), dtype=complex)
        for blk in range(p.n_blocks):
            k = p.block_src(blk)
            arr[p.block_freq(blk), w.survey.rec_offsets[k]:w.survey.rec_offsets[k + 1]] = d[blk]
        f.set_observed(i, arr)
    f.forward(P.default_opts())
    Ks = [kkt.KKT(p, w.gamma_start.ravel(), d, EPS, include_Ls_n=True) for w, p, d in zip(wls, probs, d_obs)]
    yield P, f, wls, probs, Ks
    f.close()


def _smooth_vectors(K, w, m, seed):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(m):
        v = FI.smooth(g.standard_normal((w.grid.nz, w.grid.nx)), 3.0).ravel()
        out.append(v / np.linalg.norm(v))
    return out


@pytest.fixture(scope="module")
def pairs(setup):
    """Three exact pairs (s, H s) on instance 0 and two on instance 1, from the
    oracle's matrix-free Hessian; concatenated rows for the library (zeros on
    the other instance), per-instance lists for the oracle."""
    P, f, wls, probs, Ks = setup
    per = []
    for i, (K, w) in enumerate(zip(Ks, wls)):
        per.append([(s, K.normal_matvec(s)) for s in _smooth_vectors(K, w, 3 - i, 40 + i)])
    nc = [K.Nc for K in Ks]
    S, Y = [], []
    order = [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2)]           # interleaved instances, oldest first
    for i, j in order:
        s = np.zeros(sum(nc)); y = np.zeros(sum(nc))
        o = sum(nc[:i])
        s[o:o + nc[i]], y[o:o + nc[i]] = per[i][j]
        S.append(s); Y.append(y)
    return np.array(S), np.array(Y), per


def _pack(parts):
    du = np.concatenate([p[0].ravel() for p in parts])
    lm = np.concatenate([p[2].ravel() for p in parts])
    ds = np.concatenate([p[1].ravel() for p in parts])
    return np.concatenate([du.view(np.float64), lm.view(np.float64), ds])


def _unpack(Ks, x):
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


def test_hessian_apply_matches_oracle(setup):
    P, f, wls, probs, Ks = setup
    vs = [_smooth_vectors(K, w, 1, 7 + i)[0] for i, (K, w) in enumerate(zip(Ks, wls))]
    hv, st = f.hessian_apply(np.concatenate(vs), P.default_opts(eps=EPS))
    o = 0
    for K, v in zip(Ks, vs):
        ref = K.normal_matvec(v)
        assert _rel(hv[o:o + K.Nc], ref) < 1e-6, _rel(hv[o:o + K.Nc], ref)
        o += K.Nc
    # the device-buffer form gives the same product
    hv2, _ = f.hessian_apply(torch.from_numpy(np.concatenate(vs)).cuda(), P.default_opts(eps=EPS))
    assert _rel(hv2.cpu().numpy(), hv) < 1e-12


def test_hblock_preconditioner_matches_oracle(setup, pairs):
    P, f, wls, probs, Ks = setup
    S, Y, per = pairs
    f.hblock_set(S, Y)
    opts = P.default_opts(eps=EPS, inner_iters=4, hblock=1)
    rng = np.random.default_rng(11)
    parts = [(rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N)), rng.standard_normal(K.Nc),
              rng.standard_normal((K.B, K.N)) + 1j * rng.standard_normal((K.B, K.N))) for K in Ks]
    z = f.apply_precond(torch.from_numpy(_pack(parts)).cuda(), opts).cpu().numpy()
    got = _unpack(Ks, z)
    for K, w, p, pr, g, pp in zip(Ks, wls, probs, parts, got, per):
        hs = {fi: mg.Hierarchy(w.grid, p.omegas[fi], p.gamma_pad(w.gamma_start.ravel()), shift=opts.shift_beta,
                               nu1=opts.nu1, nu2=opts.nu2, wj=opts.omega_jac, cycle=opts.mg_cycle,
                               sigma_cap=opts.sigma_cap, wdepth=opts.mg_wdepth) for fi in range(w.survey.n_freq)}

        def inner(b, rhs, adj):
            return mg.inner_solve(K.A[p.block_freq(b)], hs[p.block_freq(b)], rhs, 4, adj)[0]
        ref = K.unpack(K.precond(K.pack(*pr), inner, hblock=lambda t: lbfgs.two_loop(t, pp, 1.0 / EPS)))
        for a, r in zip(g, ref):
            assert _rel(a, r) < 1e-8, _rel(a, r)
        # the H block changed the control part (not the eps I result)
        ref0 = K.unpack(K.precond(K.pack(*pr), inner))
        assert _rel(ref0[1], ref[1]) > 1e-3
    # complex64 application agrees with complex128 to single precision
    z32 = f.apply_precond(torch.from_numpy(_pack(parts)).float().cuda(), opts).double().cpu().numpy()
    assert _rel(z32, z) < 1e-4
    f.hblock_set()


@pytest.fixture(scope="module")
def direct_updates(setup):
    P, f, wls, probs, Ks = setup
    return [K.delta_s(K.solve_direct()) for K in Ks]


@pytest.mark.parametrize("prec", [1, 0])
def test_kkt_solve_with_hblock_matches_direct(setup, direct_updates, prec):
    """Pairs from the library's own Hessian product at the current model (the
    way a Newton driver builds them); the solve reaches the direct solution."""
    P, f, wls, probs, Ks = setup
    base = P.default_opts(eps=EPS, precision=prec, tol=1e-7, inner_iters=6)
    S = []
    for i, (K, w) in enumerate(zip(Ks, wls)):
        for v in _smooth_vectors(K, w, 2, 60 + i):
            s = np.zeros(sum(k.Nc for k in Ks))
            o = sum(k.Nc for k in Ks[:i])
            s[o:o + K.Nc] = v
            S.append(s)
    Y = [f.hessian_apply(s, base)[0] for s in S]
    f.hblock_set(np.array(S), np.array(Y))
    ds, st = f.kkt_solve(P.default_opts(eps=EPS, precision=prec, tol=1e-7, inner_iters=6, hblock=1))
    assert st["rel_res"] <= 1e-7
    o = 0
    for K, ref in zip(Ks, direct_updates):
        n = K.Nc
        assert _rel(ds[o:o + n], ref) < 1e-5, _rel(ds[o:o + n], ref)
        o += n
    f.hblock_set()


def test_hblock_graph_replay_equals_direct_launches(setup, pairs):
    P, f, wls, probs, Ks = setup
    S, Y, _ = pairs
    f.hblock_set(S, Y)
    res = []
    for g in (1, 0):
        ds, st = f.kkt_solve(P.default_opts(eps=EPS, tol=1e-7, inner_iters=6, hblock=1, use_graph=g))
        res.append((ds, st["outer_iters"]))
    assert res[0][1] == res[1][1]
    assert _rel(res[0][0], res[1][0]) < 1e-12
    f.hblock_set()


def test_hblock_refusals_and_empty_set(setup, pairs):
    P, f, wls, probs, Ks = setup
    S, Y, _ = pairs
    with pytest.raises(P.FwiError):
        f.hblock_set(S[:1], -Y[:1])                         # s^T y < 0
    with pytest.raises(P.FwiError):
        f.hblock_set(np.tile(S[:1], (9, 1)), np.tile(Y[:1], (9, 1)))   # more than FWI_HBLOCK_MAX
    # no pairs: hblock = 1 is the paper's eps I block, bit for bit
    f.hblock_set()
    v = torch.from_numpy(np.random.default_rng(3).standard_normal(f.layout()["kkt_elems"])).cuda()
    z0 = f.apply_precond(v, P.default_opts(eps=EPS, inner_iters=2))
    z1 = f.apply_precond(v, P.default_opts(eps=EPS, inner_iters=2, hblock=1))
    assert torch.equal(z0, z1)
