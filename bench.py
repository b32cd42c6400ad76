#!/usr/bin/env python
"""Benchmark: one full-space Gauss-Newton step (Sec. 3-5) on the
Marmousi-shaped synthetic workload (401x141 core, h = 20 m, 20-node absorbing
layer, 40 surface sources x 3/5/7 Hz = 120 Helmholtz blocks, 401 receivers).

A step = set-up of the multigrid hierarchy, forward modelling of all blocks
(FP64-refined), data residual, the KKT solve to 1e-6 relative residual with the
inexact block-triangular preconditioner (complex64 bulk, FP64 refinement), and
the model update.  Timed steps walk the workload's 5-step Gauss-Newton
trajectory from the starting model (reset after every 5 steps).  Observed data
come from the library's own forward modelling at the true model (untimed
set-up).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line (rank 0).  --impl reference times the CPU oracle (exact
block solves by sparse LU, i.e. the paper's GMRes-full) on whole steps of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Newton-step KKT solve time to 1e-6 residual; Krylov iters/s; stencil HBM GB/s"
EPS = 1e-1            # regulariser weight on the relative model: the oracle's exact-preconditioner
                      # GMRES(30) needs 13 iterations here (the paper's Table 1: 16)
WORKLOAD = "marmousi_shaped_401x141_h20_pml20_40src_3-5-7Hz_120blocks"
INCLUDE_LS_N = 0      # regulariser on the update only (Levenberg-Marquardt damping), as in the paper's
                      # multi-frequency experiment: with the -L s_n term, eps = 0.1 on the absolute model
                      # pulls the model towards zero and a 5-step trajectory diverges after step 1


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def replica_throughput(seconds: float, steps: int, device: str = "cuda"):
    """Whole-job throughput of N independent replicas (one per rank, each doing
    ``steps`` Newton steps of the same workload): the timed region of the job
    is the slowest rank's, so the seconds are reduced by MAX over the process
    group (when one is initialised) and value = ranks / (max seconds / steps).
    Returns (value, per-step seconds)."""
    import torch
    import torch.distributed as dist
    ws = 1
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = t.item()
    per_step = seconds / steps
    return ws / per_step, per_step


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, gpu_index: int = 0):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx = float(s[2])
                for n, v in zip(names, s[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# dram__bytes_read.sum + dram__bytes_write.sum of the level-0 smoother launches
# per byte of the pass itself (b and the result, plus x unless it starts from
# zero, plus r, v and the old p when it forms the p update), from the ncu
# captures of its three variants summarised under profiles/ (the p-update pass
# is k_jacobi2_stage, the others k_jacobi2_march), weighted as the timed
# forward solves launch them (per BiCGStab iteration: one with the p update,
# one from zero, two from x): (356.9 + 115.5 + 2 x 206.8) MB over
# (383.2 + 153.3 + 2 x 229.9) MB.  None once a kernel changes.
TRAFFIC_PER_FUSED_BYTE = (356.9 + 115.5 + 2 * 206.8) / (383.2 + 153.3 + 2 * 229.9)
# warp instructions of one k_coarse_cycle<float, 0, 512> launch on the
# benchmark workload (120 blocks, levels 110x45 .. 13x5, W(2,2) to level 2),
# smsp__inst_executed.sum of the ncu capture summarised under profiles/; the
# kernel is latency-bound, so its roofline is the instruction issue rate of
# the chip (152 SMs x 4 schedulers x the SM clock).  None once it changes.
COARSE_CYCLE_WARP_INSTS = 26.98e6


def _roofline(ms, nbytes, n, peaks, fused_bytes=None):
    """Roofline of the level-0 two-sweep smoother from the library's live
    timing of its direct launches: achieved = algorithmic bytes per launch
    (the scope table's 24 B per node and damped-Jacobi sweep for complex64:
    x, b and the result, two sweeps per launch, 40 B per node when the first
    sweep starts from zero) over the average launch duration (CUDA events on
    the launching stream)."""
    peak = peaks.get("hbm_gbs")
    src = "MEASURED_PEAKS.json hbm_gbs (measured)"
    if not peak:
        peak, src = 6800.0, "fallback 6.8 TB/s"
    if not n or ms <= 0:
        return None
    ach = nbytes / (ms / 1e3) / 1e9
    per_launch = nbytes / n
    out = {"kernel": "k_jacobi2_march / k_jacobi2_stage <float> at level 0 (two fused damped-Jacobi sweeps of "
                     "the shifted 5-point PML stencil, all blocks, all three passes)",
           "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "peak_source": src, "launches_timed": n, "avg_launch_us": ms / n * 1e3,
           "algorithmic_bytes_per_launch": per_launch,
           "accounting": "24 B per node and sweep (x, b, result), 2 sweeps per launch; 40 B per node from zero"}
    if fused_bytes:
        fpl = fused_bytes / n
        out["fused_pass_bytes_per_launch"] = fpl
        out["fused_pass_gbs"] = fused_bytes / (ms / 1e3) / 1e9
        out["traffic"] = TRAFFIC_PER_FUSED_BYTE * fpl if TRAFFIC_PER_FUSED_BYTE else None
    else:
        out["traffic"] = None
    return out


def run_inner_case(args):
    """Profiling case: batched inner solves (BiCGStab + multigrid) on all 120
    blocks of the benchmark workload, without the KKT basis (about 2 GB)."""
    import numpy as np
    import torch
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    wl = _workload()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    f = P.FWI([wl.grid], stream=stream.cuda_stream)
    f.set_survey(0, wl.survey)
    f.set_model(0, wl.gamma_start)
    opts = P.default_opts(inner_iters=4)
    n = f.layout()["field_elems"]
    g = np.random.default_rng(0)
    b = torch.from_numpy((g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)).cuda()
    for _ in range(args.warmup):
        f.inner_solve(b, opts)
    torch.cuda.synchronize()
    f.stencil_timer(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f.inner_solve(b, opts)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    ms, nbytes, cnt, pb = f.stencil_timer(0, with_pass=True)
    print(json.dumps({"case": "inner", "inner_iters": 4, "s_per_solve": dt,
                      "roofline": _roofline(ms, nbytes, cnt, _peaks(), pb)}))


def _setup_ctx(P, wls, opts, stream):
    """Context over one or more workloads with synthetic data from the
    library's forward modelling at the true models (untimed)."""
    f = P.FWI([w.grid for w in wls], stream=stream.cuda_stream)
    for i, w in enumerate(wls):
        f.set_survey(i, w.survey)
        f.set_model(i, w.gamma_true)
    d, _, _ = f.forward(opts, want_data=True)
    for i, w in enumerate(wls):
        f.set_observed(i, d[i])
        f.set_model(i, w.gamma_start)
    return f


def run_extra_case(args):
    """Other workloads of the scope table, one JSON line each (not the headline):
      batch3a   1024 blocks (256 sources x 2/4/6/8 Hz, 401x141) in one batch
      batch3b   8 instances of uneven grids x 32 sources x 2/4/6/8 Hz
      large     1601x561 h=5 m, 128 sources, one frequency (4 Hz)
      autograd  801x281 h=10 m, 64 sources, 6 Hz: misfit + gradient through
                torch.autograd, with central-difference checks
      tradeoff  the benchmark workload: one KKT solve per inner-iteration count
                (2 .. 48 BiCGStab iterations per block solve, W to level 2),
                outer FGMRES iterations against time: the inexactness
                trade-off of the preconditioner's block solves
      rsgn      the benchmark workload (401x141, 120 blocks): one reduced-space
                Gauss-Newton step (normal equations by CG, two refined block
                solves per CG iteration), capped at ``--max-outer`` CG
                iterations, next to one full-space step from the same model
    batch3a/3b/large run one Newton step with a cap of ``--max-outer`` outer
    iterations and report throughput (outer and inner iterations per second)."""
    import numpy as np
    import torch
    import fwi_inputs as FI
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    opts = P.default_opts(eps=args.eps or EPS, inner_iters=args.inner_iters or 8, include_Ls_n=INCLUDE_LS_N)
    if args.case == "batch3a":
        wls = [FI.batching_workload()]
    elif args.case == "batch3b":
        wls = FI.uneven_workloads()
    elif args.case == "large":
        wls = [FI.large_workload(freqs=(4.0,))]
    elif args.case in ("rsgn", "tradeoff"):
        wls = [_workload()]
    else:
        wls = [FI.autograd_workload()]
    if args.case not in ("rsgn", "tradeoff"):
        from paper_2204_06489_gb300.autotune import auto_wdepth
        opts.mg_wdepth = auto_wdepth([w.grid for w in wls], [w.survey.freqs_hz for w in wls],
                                     [w.gamma_start for w in wls])
    t0 = time.perf_counter()
    f = _setup_ctx(P, wls, opts, stream)
    t_setup = time.perf_counter() - t0
    lay = f.layout()
    out = {"case": args.case, "workloads": [w.name for w in wls], "blocks": lay["n_blocks"],
           "mg_wdepth": opts.mg_wdepth, "inner_iters": opts.inner_iters,
           "field_complex": lay["field_elems"], "setup_s": t_setup}
    if args.case == "autograd":
        from scipy.ndimage import gaussian_filter
        from paper_2204_06489_gb300.autograd import misfit
        w = wls[0]
        g0 = torch.tensor(w.gamma_start, dtype=torch.float64, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phi = misfit(g0, f, mode="recompute", opts=opts)
        phi.backward()
        torch.cuda.synchronize()
        out["forward_backward_s"] = time.perf_counter() - t0
        grad = g0.grad.detach().cpu().numpy()
        errs = []
        for seed in range(args.fd_dirs):
            dirn = gaussian_filter(np.random.default_rng(seed).standard_normal(grad.shape), 10.0)
            dirn *= 0.003 * w.gamma_start.mean() / np.abs(dirn).max()
            with torch.no_grad():
                fp = misfit(torch.tensor(w.gamma_start + dirn, device="cuda"), f, opts=opts).item()
                fm = misfit(torch.tensor(w.gamma_start - dirn, device="cuda"), f, opts=opts).item()
            an = float(np.sum(grad * dirn))
            errs.append(abs((fp - fm) / 2 - an) / abs(an))
        out.update(misfit=phi.item(), fd_rel_err_max=max(errs), fd_directions=len(errs))
    elif args.case == "tradeoff":
        from paper_2204_06489_gb300.autotune import tune_kkt
        f.set_model(0, wls[0].gamma_start)
        f.forward(opts, want_data=False)
        o = P.Opts.from_buffer_copy(opts)
        o.max_outer = args.max_outer
        _, table = tune_kkt(f, o, (2, 4, 6, 8, 12, 16, 24, 48), (2,), (30,))
        out["sweep"] = [{"inner_solver": "bicgstab+multigrid", "inner_iters": n, "kkt_s": round(t, 3), "outer": k,
                         "converged": ok} for n, wd, rs, t, k, ok, _, _, _ in table]
        # the paper's incomplete-LU block approximation (zero fill on the GPU):
        # applied once as A~, and as the preconditioner of BiCGStab
        for solver, iters in ((2, 1), (1, 4), (1, 8), (1, 16)):
            oi = P.Opts.from_buffer_copy(o)
            oi.inner_solver = solver
            oi.inner_iters = iters
            print(f"tradeoff: inner_solver {solver}, {iters} iterations", file=sys.stderr, flush=True)
            f.kkt_solve(oi, allow_noconv=True) if solver == 2 else None   # builds the factors (untimed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = f.kkt_solve(oi, allow_noconv=True)
            torch.cuda.synchronize()
            out["sweep"].append({"inner_solver": "ilu0 once" if solver == 2 else "bicgstab+ilu0",
                                 "inner_iters": iters if solver == 1 else 0,
                                 "kkt_s": round(time.perf_counter() - t0, 3), "outer": st["outer_iters"],
                                 "converged": st["rel_res"] <= oi.tol})
    elif args.case == "rsgn":
        o = P.Opts.from_buffer_copy(opts)
        o.max_outer = args.max_outer
        res = {}
        for name, step in (("fsgn", f.newton_step), ("rsgn", f.rsgn_step)):
            f.set_model(0, wls[0].gamma_start)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ds, st = step(o if name == "rsgn" else opts, allow_noconv=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            res[name] = {"step_s": dt, "iters": st["outer_iters"], "rel_res": st["rel_res"],
                         "forward_ms": st["t_forward_ms"], "solve_ms": st["t_solve_ms"],
                         "s_per_iter": st["t_solve_ms"] / 1e3 / max(st["outer_iters"], 1)}
            res[name + "_ds"] = ds
        dk, dr = res.pop("fsgn_ds"), res.pop("rsgn_ds")
        res["rel_diff_ds"] = float(np.linalg.norm(dr - dk) / np.linalg.norm(dk))
        out.update(res)
    else:
        o = P.Opts.from_buffer_copy(opts)
        o.max_outer = args.max_outer
        f.stencil_timer(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ds, st = f.newton_step(o, allow_noconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ms, nbytes, cnt, pb = f.stencil_timer(0, with_pass=True)
        converged = st["rel_res"] <= o.tol and st["fwd_rel_res"] <= o.fwd_tol
        out.update(converged=converged, newton_step_s=dt, outer_iters=st["outer_iters"], rel_res=st["rel_res"],
                   fwd_rel_res=st["fwd_rel_res"], forward_ms=st["t_forward_ms"], kkt_ms=st["t_solve_ms"],
                   roofline=_roofline(ms, nbytes, cnt, _peaks(), pb))
        if converged:
            out.update(krylov_iters_per_s=st["outer_iters"] / (st["t_solve_ms"] / 1e3),
                       inner_block_iters_per_s=st["inner_iters"] / dt)
        else:
            out["note"] = "not converged: no throughput is reported for an unconverged solve"
    print(json.dumps(out))
    f.close()


def run_kkt_case(args):
    """Profiling case: the KKT-side kernels (KKT product, coupling reductions,
    FGMRES multi-dots and updates) on the benchmark workload: set-up, forward
    modelling, and one KKT solve stopped after ``--max-outer`` FGMRES
    iterations (a truncated solve: not a benchmark value)."""
    import torch
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    wl = _workload()
    opts = P.default_opts(eps=EPS, inner_iters=args.inner_iters or 12, include_Ls_n=INCLUDE_LS_N,
                          max_outer=args.max_outer, use_graph=0 if args.no_graph else 1)
    f = _setup_ctx(P, [wl], opts, stream)
    f.forward(opts, want_data=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = f.kkt_solve(opts, allow_noconv=True)
    torch.cuda.synchronize()
    print(json.dumps({"case": "kkt", "outer_iters": st["outer_iters"], "rel_res": st["rel_res"],
                      "s": time.perf_counter() - t0}))
    f.close()


def run_epsrule_case(args):
    """The regulariser rule eps = alpha * lambda_max(Re J~^H W^T W J~), alpha =
    1e-2, lambda_max from 10 power iterations on the matrix-free Gauss-Newton
    operator (fwi_normal_lambda_max) at the starting model of the benchmark
    workload; then one Newton step at that eps and one at the headline eps,
    with their FGMRES iterations and times (one JSON line)."""
    import torch
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    wl = _workload()
    opts = P.default_opts(eps=EPS, inner_iters=args.inner_iters or 12, max_outer=args.max_outer,
                          include_Ls_n=INCLUDE_LS_N)
    f = _setup_ctx(P, [wl], opts, stream)
    f.forward(opts, want_data=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, _ = f.normal_lambda_max(opts, iters=10)
    t_lam = time.perf_counter() - t0
    eps_rule = 1e-2 * lam
    out = {"case": "epsrule", "lambda_max": lam, "power_iters": 10, "lambda_s": round(t_lam, 2),
           "alpha": 1e-2, "eps_rule": eps_rule, "steps": []}
    # the block solves' accuracy tied to eps: the autotuner picks the inner
    # iteration count at each eps (one KKT solve per candidate, untimed)
    from paper_2204_06489_gb300.autotune import tune_kkt
    chosen = {}
    for eps, cands in ((eps_rule, (16, 24, 32, 48, 64)), (EPS, (4, 6, 8, 12, 16))):
        o = P.Opts.from_buffer_copy(opts)
        o.eps = eps
        f.set_model(0, wl.gamma_start)
        f.forward(o, want_data=False)
        best, table = tune_kkt(f, o, cands, (None,), (None,))
        chosen[eps] = best.inner_iters
        out.setdefault("autotune", []).append({"eps": eps, "table": [
            {"inner_iters": n, "s": round(t, 3), "outer": k, "ok": ok} for n, wd, rs, t, k, ok, _, _, _ in table]})
    for eps in (eps_rule, EPS):
        o = P.Opts.from_buffer_copy(opts)
        o.eps = eps
        o.inner_iters = chosen[eps]
        f.set_model(0, wl.gamma_start)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ds, st = f.newton_step(o, allow_noconv=True)
        torch.cuda.synchronize()
        out["steps"].append({"eps": eps, "inner_iters": o.inner_iters,
                             "step_s": round(time.perf_counter() - t1, 3), "outer_iters": st["outer_iters"],
                             "rel_res": st["rel_res"], "converged": st["rel_res"] <= o.tol,
                             "kkt_ms": st["t_solve_ms"]})
    print(json.dumps(out))
    f.close()


def run_hblock_case(args):
    """The quasi-Newton H block (L-BFGS in place of L = eps I; Sec. 5 after eq.
    precond, Sec. 7) against the paper's block along the benchmark's 5-step
    trajectory.  After each step the pair (ds~_k, H~(s_{k+1}) ds~_k) is formed
    with the library's Hessian product at the new model (one forward and one
    adjoint refined solve per block, timed as pair_s); the newest 5 pairs are
    kept.  At the headline eps (inner iterations --inner-iters, default 6) and,
    with --eps, at another eps (e.g. the epsrule case's eps_rule, with the inner
    iterations that case picked).  One JSON line."""
    import numpy as np
    import torch
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    wl = _workload()
    eps = args.eps or EPS
    opts = P.default_opts(eps=eps, inner_iters=args.inner_iters or 6, max_outer=args.max_outer,
                          include_Ls_n=INCLUDE_LS_N)
    f = _setup_ctx(P, [wl], opts, stream)
    gref = float(np.mean(wl.gamma_true))
    out = {"case": "hblock", "eps": eps, "inner_iters": opts.inner_iters, "pairs_kept": 5, "runs": []}
    for hb in (0, 1):
        o = P.Opts.from_buffer_copy(opts)
        o.hblock = hb
        f.set_model(0, wl.gamma_start)
        f.hblock_set()
        S, Y, rows = [], [], []
        prev = None
        for k in range(NEWTON_STEPS):
            pair_s = 0.0
            if hb and prev is not None:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                f.forward(o, want_data=False)
                y, _ = f.hessian_apply(prev, o)
                torch.cuda.synchronize()
                pair_s = time.perf_counter() - t0
                if float(prev @ y) > 0.0:
                    S.append(prev); Y.append(y)
                    S, Y = S[-5:], Y[-5:]
                    f.hblock_set(np.array(S), np.array(Y))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ds, st = f.newton_step(o, allow_noconv=True)
            torch.cuda.synchronize()
            rows.append({"newton_step": k + 1, "pairs": len(S), "outer_iters": st["outer_iters"],
                         "kkt_ms": round(st["t_solve_ms"], 1), "step_s": round(time.perf_counter() - t1, 3),
                         "pair_s": round(pair_s, 3), "rel_res": st["rel_res"],
                         "converged": st["rel_res"] <= o.tol, "misfit": st["misfit"]})
            prev = np.asarray(ds, dtype=np.float64).ravel() / gref
        out["runs"].append({"hblock": "L-BFGS" if hb else "eps I", "steps": rows,
                            "total_s": round(sum(r["step_s"] + r["pair_s"] for r in rows), 3),
                            "outer_total": sum(r["outer_iters"] for r in rows)})
        print(json.dumps(out["runs"][-1]), file=sys.stderr, flush=True)
    f.hblock_set()
    print(json.dumps(out))
    f.close()


def _workload():
    import fwi_inputs as FI
    return FI.marmousi_shaped_workload()


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_step(workers: int = 0, n_src: int = 40, freqs=(3.0, 5.0, 7.0)):
    """The oracle as it stands, on the host cores: one whole Gauss-Newton step
    of the benchmark workload (by default all 120 blocks) with the paper's
    GMRes-full, i.e. GMRES(30) with the exact block-triangular preconditioner
    (sparse LU block solves), eps and tolerance as the GPU step.  Timed: LU
    factorisations, forward modelling of every block, the KKT solve to 1e-6
    and the model update.  ``workers`` > 0 spreads the independent block
    solves over a spawned process pool (one BLAS thread each); 0 runs
    everything in this process.  Observed data come from the oracle's forward
    modelling at the true model (untimed)."""
    import numpy as np
    import fwi_inputs as FI
    from oracle import fwi, helmholtz, kkt, krylov
    from oracle.pool import BlockPool
    wl = FI.marmousi_shaped_workload(n_src=n_src, freqs=freqs)
    prob = fwi.Problem.create(wl.grid, wl.survey, wl.gamma_start)
    src = np.array([helmholtz.source_vector(wl.grid, int(wl.survey.src_ix[prob.block_src(b)]),
                                            int(wl.survey.src_iz[prob.block_src(b)]),
                                            complex(wl.survey.src_amp[prob.block_src(b)]))
                    for b in range(prob.n_blocks)])
    s0 = wl.gamma_start.ravel()
    if workers > 0:
        ptrue = BlockPool(prob, wl.gamma_true.ravel(), workers)
        d = fwi.sample(prob, ptrue.solve(src, False))
        ptrue.close()
        pool = BlockPool(prob, s0, workers)
        pool.warm()
    else:
        d = fwi.sample(prob, fwi.forward(prob, wl.gamma_true.ravel()))
        prob._lu.clear()
        pool = None
    t0 = time.perf_counter()
    if pool is not None:
        u = pool.solve(src, False)
        K = kkt.KKT(prob, s0, d, EPS, include_Ls_n=bool(INCLUDE_LS_N), u_n=u)
        pre = lambda v: K.precond(v, inner_batch=pool.solve)   # noqa: E731
    else:
        K = kkt.KKT(prob, s0, d, EPS, include_Ls_n=bool(INCLUDE_LS_N))
        pre = K.precond
    x, info = krylov.fgmres(K.matvec, K.rhs(), pre, restart=30, tol=1e-6, max_iter=300)
    s1 = s0 + K.delta_s(x)
    dt = time.perf_counter() - t0
    if pool is not None:
        pool.close()
    mode = f"process pool of {workers} workers over the blocks" if workers else "one process"
    return {"seconds": dt, "iters": info["iters"], "true_relres": info["true_relres"], "blocks": prob.n_blocks,
            "threads": workers if workers else 1, "mode": mode, "update_norm": float(np.linalg.norm(s1 - s0))}


def cpu_baseline(workers: int | None = None):
    """cpu_baseline of the bench line: the whole 120-block Gauss-Newton step of
    the oracle (no sample scaling), exact block solves spread over one process
    per host core."""
    w = _cores() if workers is None else workers
    r = oracle_step(workers=w)
    return {"value": 1.0 / r["seconds"], "unit": "Newton-step KKT solves/s", "cores": r["threads"], "kind": "oracle",
            "sample": (f"the whole benchmark step: 401x141 grid, {r['blocks']} blocks (40 sources x 3/5/7 Hz), "
                       f"LU factorisation + forward + exact-preconditioner GMRES(30) to 1e-6 "
                       f"({r['iters']} iterations, true residual {r['true_relres']:.1e}) + update, "
                       f"{r['mode']}, {r['seconds']:.1f} s; no scaling"),
            "seconds": r["seconds"], "iters": r["iters"]}


def run_reference(args):
    """The reference arm: the oracle (the paper's GMRes-full on the host cores)
    on the benchmark workload.  One whole Newton step of the oracle takes tens
    of seconds, so the arm times min(steps, 2) whole steps after no warm-up
    (the oracle has no warm-up effects beyond process start, which is outside
    the timed region) and says so in the line."""
    ws, rank = _dist()
    if rank != 0:
        return
    n = max(1, min(args.steps, 2))
    runs = [oracle_step(workers=_cores()) for _ in range(n)]
    mean = sum(r["seconds"] for r in runs) / n
    v = 1.0 / mean
    r = runs[-1]
    sample = (f"whole steps of the benchmark workload (120 blocks), {r['mode']}, GMRES(30) with the exact "
              f"preconditioner to 1e-6 ({r['iters']} iterations); {n} timed step(s) of the requested "
              f"{args.steps} (each whole step takes {mean:.0f} s), no warm-up")
    cb = {"value": v, "unit": "Newton-step KKT solves/s", "cores": r["threads"], "kind": "oracle", "sample": sample}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton-step KKT solves/s",
                      "n_gpus": ws, "steps": n, "warmup": 0, "ms_per_step": mean * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
                      "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": "Newton-step KKT solves/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}))


def cpu_baseline_fields(r):
    return {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}


NEWTON_STEPS = 5       # Gauss-Newton steps of the workload's trajectory (the model is reset after them)


def _kernel_table(prof, peak, wall_ms):
    """Rows of the library's kernel profile of one step, largest total time
    first: launches, total and average device time, algorithmic bytes per
    launch, achieved GB/s and its fraction of the measured HBM bandwidth."""
    rows = []
    tot = sum(r["ms"] for r in prof["rows"])
    for r in sorted(prof["rows"], key=lambda r: -r["ms"]):
        name = r["kernel"] + (f"[L{r['level']}]" if r["level"] >= 0 and r["kernel"] != "k_coupling_reduce" else
                              (f"[mode {r['level']}]" if r["kernel"] == "k_coupling_reduce" else ""))
        gbs = r["bytes"] / (r["ms"] / 1e3) / 1e9 if r["ms"] > 0 and r["bytes"] > 0 else None
        rows.append({"kernel": name, "launches": r["launches"], "ms": round(r["ms"], 3),
                     "share": round(r["ms"] / tot, 4) if tot else None,
                     "avg_us": round(r["ms"] / r["launches"] * 1e3, 2),
                     "bytes_per_launch": round(r["bytes"] / r["launches"]) if r["bytes"] else 0,
                     "gbs": round(gbs, 1) if gbs else None, "frac": round(gbs / peak, 3) if gbs else None})
    return {"kernel_ms": round(tot, 3), "gap_ms": round(prof["gap_ms"], 3), "wall_ms": round(wall_ms, 3),
            "rows": rows}


def run_newton(args):
    """The headline line: Gauss-Newton steps of the 120-block workload.  Each
    timed step is one step of the workload's 5-step trajectory (steps 1-5 from
    the starting model, then the model is reset), so K = 5, 10, ... times whole
    trajectories; inputs are resident in HBM; CUDA events on the context's
    stream give per-step device times."""
    import ctypes as C
    import numpy as np
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2204_06489_gb300 as P
    P.load(build_if_missing=True)
    wl = _workload()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    f = P.FWI([wl.grid], stream=stream.cuda_stream)
    f.set_survey(0, wl.survey)
    opts = P.default_opts(eps=args.eps or EPS, precision=args.precision, include_Ls_n=INCLUDE_LS_N)
    if args.inner_iters:
        opts.inner_iters = args.inner_iters
    if args.restart:
        opts.restart = args.restart
    if args.profile_outer:
        opts.max_outer = args.profile_outer
    # synthetic observed data: the library's forward modelling at the true model
    f.set_model(0, wl.gamma_true)
    d_true, _, _ = f.forward(opts)
    f.set_observed(0, d_true[0])
    tuned = None
    if not args.inner_iters:
        # untimed set-up: pick the inner iteration count by timing one KKT solve each
        from paper_2204_06489_gb300.autotune import tune_kkt
        f.set_model(0, wl.gamma_start)
        f.forward(opts, want_data=False)
        opts, table = tune_kkt(f, opts, (4, 6, 8, 12, 16), (1, 2), (30,), nus=(1, 2))
        # second stage at the chosen schedule: strip height x coarse-cycle CTA size, scored by
        # time per FGMRES iteration (the layout changes no arithmetic)
        opts, table2 = tune_kkt(f, opts, (opts.inner_iters,), (None,), (None,), (8, 16, 32), (512, 1024),
                                per_iteration=True)
        tuned = [{"inner_iters": n, "wdepth": wd, "restart": rs, "strip_rows": sr, "coarse_threads": ct,
                  "nu": nu, "s": round(t, 3), "outer": o, "ok": ok}
                 for n, wd, rs, t, o, ok, sr, ct, nu in table + table2]
    g0 = torch.from_numpy(wl.gamma_start).cuda()
    ds_dev = torch.zeros(wl.grid.nx * wl.grid.nz, dtype=torch.float64, device="cuda")

    def step_device(k, o=None):
        st = P.api.Stats()
        if k % NEWTON_STEPS == 0:
            f.set_model(0, g0)
        rc = f._L.fwi_newton_step(f._h, C.byref(o or opts), C.c_void_p(ds_dev.data_ptr()), 1, C.byref(st))
        f._check(rc, allow_noconv=bool(args.profile_outer))
        return st

    for k in range(args.warmup):
        step_device(k)
    torch.cuda.synchronize()
    f.stencil_timer(1)          # live CUDA-event timing of the level-0 smoother kernel
    launches0 = f._L.fwi_kernel_launches()
    clocks = Clocks(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    stats = []
    for k in range(args.steps):
        stats.append(step_device(k))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    dev_s = ev[0].elapsed_time(ev[-1]) / 1e3
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    launches = f._L.fwi_kernel_launches() - launches0
    st_ms, st_bytes, st_n, st_pass = f.stencil_timer(0, with_pass=True)
    value, per_step = replica_throughput(dev_s, args.steps)
    traj = []
    for q in range(min(NEWTON_STEPS, args.steps)):
        sel = [k for k in range(args.steps) if k % NEWTON_STEPS == q]
        traj.append({"newton_step": q + 1, "ms": round(sum(step_ms[k] for k in sel) / len(sel), 1),
                     "outer_iters": sum(stats[k].outer_iters for k in sel) / len(sel),
                     "rel_res": max(stats[k].rel_res for k in sel),
                     "misfit": stats[sel[0]].misfit})

    # end to end through the C ABI with host buffers (h2d model + data, d2h
    # update), walking the same trajectory: the host keeps the model
    g_start = np.ascontiguousarray(wl.gamma_start)
    d_host = np.ascontiguousarray(d_true[0])
    ds_host = np.zeros(wl.grid.nx * wl.grid.nz)
    g_host = g_start.copy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        if k % NEWTON_STEPS == 0:
            g_host = g_start.copy()
        f.set_model(0, g_host)
        f.set_observed(0, d_host)
        st = P.api.Stats()
        f._check(f._L.fwi_newton_step(f._h, C.byref(opts), ds_host.ctypes.data_as(C.c_void_p), 0, C.byref(st)),
                 allow_noconv=bool(args.profile_outer))
        g_host = g_host + ds_host.reshape(g_host.shape)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps

    peaks = _peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    extras = {}
    if not args.no_extras and ws == 1:
        step1 = [step_ms[k] for k in range(args.steps) if k % NEWTON_STEPS == 0]
        # (a) the plain complex128 GPU form of the same method, same tolerance,
        # step 1 of the trajectory (one untimed warm-up step first)
        o128 = P.Opts.from_buffer_copy(opts)
        o128.precision = 0
        step_device(0, o128)
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        st128 = step_device(0, o128)
        e_b.record(stream)
        torch.cuda.synchronize()
        ms128 = e_a.elapsed_time(e_b)
        extras["c128"] = {"ms_step1": round(ms128, 1), "outer_iters": st128.outer_iters,
                          "rel_res": st128.rel_res, "mixed_ms_step1": round(sum(step1) / len(step1), 1),
                          "mixed_speedup": round(ms128 / (sum(step1) / len(step1)), 2)}
        # (b) per-kernel table of one whole trajectory (steps 1-5) with direct
        # launches (no graph replay), CUDA events around every launch
        op = P.Opts.from_buffer_copy(opts)
        op.use_graph = 0
        for k in range(NEWTON_STEPS):                       # warm-up of the direct path
            step_device(k, op)
        f.kernel_profile(1)
        e_a.record(stream)
        stp = [step_device(k, op) for k in range(NEWTON_STEPS)]
        e_b.record(stream)
        torch.cuda.synchronize()
        prof = f.kernel_profile(0)
        kt = _kernel_table(prof, peak, e_a.elapsed_time(e_b))
        for r in kt["rows"]:
            r["launches_per_step"] = round(r["launches"] / NEWTON_STEPS, 1)
        traj_ms = sum(step_ms[k] for k in range(min(args.steps, NEWTON_STEPS)))
        kt["outer_iters"] = [s.outer_iters for s in stp]
        kt["note"] = (f"the {NEWTON_STEPS}-step trajectory with direct launches (no graph replay); kernel_ms = sum of "
                      "per-launch event times; gap_share_of_graph_steps = 1 - kernel_ms / the timed (graph-replayed) "
                      "time of the same trajectory")
        if args.steps >= NEWTON_STEPS:
            kt["gap_share_of_graph_steps"] = round(1.0 - kt["kernel_ms"] / traj_ms, 4)
        extras["kernel_table"] = kt
        # issue-rate roofline of the shared-memory coarse cycle (the largest
        # single kernel; latency-bound, about 1 % of HBM)
        cc = [r for r in kt["rows"] if r["kernel"].startswith("k_coarse_cycle")]
        if cc and COARSE_CYCLE_WARP_INSTS:
            mhz = (ck or {}).get("sm_mhz") or 2070.0
            peak_i = 152 * 4 * mhz * 1e6 / 1e9
            ach_i = COARSE_CYCLE_WARP_INSTS / (cc[0]["avg_us"] * 1e-6) / 1e9
            extras["roofline_coarse_cycle"] = {
                "kernel": "k_coarse_cycle<float> (levels 2-5 in shared memory, one CTA per block)",
                "bound": "issue", "achieved": round(ach_i, 1), "peak": round(peak_i, 1),
                "unit": "G warp-instructions/s", "frac": round(ach_i / peak_i, 3),
                "avg_launch_us": cc[0]["avg_us"],
                "accounting": "ncu warp instructions per launch (profiles/) over the live average launch time; "
                              "peak = 152 SMs x 4 schedulers x the sampled SM clock"}
        # (c) the three forms of the Arnoldi inner products (0 FP32 runs, 1 FP64
        # products, 2 compensated Dot2), with the measured loss of orthogonality
        # of the complex64 basis (max |I - V^T V|)
        arn = []
        for fp64 in (2, 1, 0):
            oa = P.Opts.from_buffer_copy(opts)
            oa.arnoldi_dots = fp64
            oa.check_orth = 1
            f.set_model(0, g0)
            f.forward(oa, want_data=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, sa = f.kkt_solve(oa, allow_noconv=True)
            torch.cuda.synchronize()
            arn.append({"arnoldi_dots": fp64, "outer_iters": sa["outer_iters"], "rel_res": sa["rel_res"],
                        "orth_loss": sa["orth_loss"], "kkt_s_with_check": round(time.perf_counter() - t1, 3)})
        extras["arnoldi"] = arn
    outer = sum(s.outer_iters for s in stats) / len(stats)
    inner = sum(s.inner_iters for s in stats) / len(stats)
    out = {"metric": METRIC, "value": value, "unit": "Newton-step KKT solves/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "c64+f64-refine" if args.precision == 1 else "c128",
           "data": "synthetic (seeded layered-faulted model; data from the library's forward modelling)",
           "config": {"workload": WORKLOAD, "blocks": 120, "grid_padded": "441x181", "eps": opts.eps,
                      "tol": 1e-6, "restart": opts.restart, "inner_iters": opts.inner_iters,
                      "include_Ls_n": INCLUDE_LS_N, "strip_rows": opts.strip_rows,
                      "coarse_threads": opts.coarse_threads, "arnoldi_dots": opts.arnoldi_dots,
                      "mg": f"W({opts.nu1},{opts.nu2}) to level {opts.mg_wdepth}, V below",
                      "steps": f"each timed step is one of the {NEWTON_STEPS} Gauss-Newton steps of the "
                               f"trajectory from the starting model (reset after {NEWTON_STEPS})",
                      "l2": "working set > L2 (packed KKT vector 153 MB, Krylov basis 9.4 GB)",
                      "parallelism": "replicas" if ws > 1 else "single GPU"},
           "outer_iters_per_step": outer, "krylov_iters_per_s": outer / per_step,
           "inner_block_iters_per_s": inner / per_step, "rel_res_max": max(s.rel_res for s in stats),
           "trajectory": traj,
           "phase_ms": {"forward": sum(s.t_forward_ms for s in stats) / len(stats),
                        "kkt_solve": sum(s.t_solve_ms for s in stats) / len(stats)},
           "forward_sweeps": sum(s.fwd_sweeps for s in stats) / len(stats), "autotune": tuned,
           "gpu_launches": int(launches),
           "roofline": _roofline(st_ms, st_bytes, st_n, peaks, st_pass),
           "clocks": ck,
           "e2e": {"value": ws / e2e_s, "unit": "Newton-step KKT solves/s",
                   "h2d_bytes_per_step": int(g_start.nbytes + d_host.nbytes),
                   "d2h_bytes_per_step": int(ds_host.nbytes)}}
    out.update(extras)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_fields(cpu_baseline())
    if rank == 0:
        print(json.dumps(out))
    f.close()
    if ws > 1:
        dist.destroy_process_group()



def main():
    import faulthandler
    faulthandler.enable()            # a native crash prints the Python stack to stderr
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the untimed extras of the headline line (complex128 form, kernel table, "
                         "Arnoldi precision comparison)")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--no-graph", action="store_true", help="profiling cases: direct launches, no graph replay")
    ap.add_argument("--case", default="newton",
                    choices=["newton", "inner", "batch3a", "batch3b", "large", "autograd", "rsgn", "tradeoff",
                             "epsrule", "kkt", "hblock"])
    ap.add_argument("--max-outer", type=int, default=60)
    ap.add_argument("--fd-dirs", type=int, default=4)
    ap.add_argument("--inner-iters", type=int, default=None)
    ap.add_argument("--restart", type=int, default=None)
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--profile-outer", type=int, default=None,
                    help="profiling runs only: cap the FGMRES iterations of the Newton step "
                         "(the step is then truncated and its number is not a benchmark value)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "inner":
        return run_inner_case(args)
    if args.case == "epsrule":
        return run_epsrule_case(args)
    if args.case == "kkt":
        return run_kkt_case(args)
    if args.case == "hblock":
        return run_hblock_case(args)
    if args.case != "newton":
        return run_extra_case(args)
    return run_newton(args)


if __name__ == "__main__":
    main()
