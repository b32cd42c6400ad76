"""Autotuner for the inner block solver's multigrid schedule.

The paper leaves the inner solver open; its speed depends on the smoother
schedule (sweeps, damping), on how deep the W-cycle goes, and on the grids and
frequencies of the batch.  ``tune_inner`` times the batched inner solve
(BiCGStab + multigrid, ``inner_iters`` iterations) for each candidate schedule
on a given right-hand side and keeps the one with the largest residual
reduction per second: rate = -ln(||b - A x|| / ||b||) / seconds.  The residual
is formed with the library's own operator (fwi_apply_helmholtz).
"""
from __future__ import annotations

import itertools
import math
import time
from typing import Iterable, Optional

from .api import FWI, Opts, default_opts


def _residual_ratio(fwi: FWI, b, x) -> float:
    import torch
    r = b - fwi.apply_helmholtz(x)
    return float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))


def tune_inner(fwi: FWI, b, base: Optional[Opts] = None, nus: Iterable[int] = (1, 2),
               omegas: Iterable[float] = (0.5, 0.6), wdepths: Iterable[int] = (1, 2, 3),
               cycles: Iterable[int] = (2,), repeats: int = 2):
    """Returns (best Opts, table of (nu, omega, wdepth, cycle, ratio, seconds, rate))."""
    import torch
    base = base if base is not None else default_opts()
    table = []
    best, best_rate = None, -math.inf
    for nu, om, wd, cy in itertools.product(nus, omegas, wdepths, cycles):
        o = Opts.from_buffer_copy(base)
        o.nu1 = o.nu2 = nu
        o.omega_jac = om
        o.mg_wdepth = wd
        o.mg_cycle = cy
        fwi.inner_solve(b, o)                      # warm-up (builds tables, buffers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(repeats):
            x = fwi.inner_solve(b, o)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / repeats
        ratio = _residual_ratio(fwi, b, x)
        rate = -math.log(max(ratio, 1e-300)) / dt if ratio < 1.0 else -math.inf
        table.append((nu, om, wd, cy, ratio, dt, rate))
        if rate > best_rate:
            best, best_rate = o, rate
    return best, table


def tune_kkt(fwi: FWI, base: Optional[Opts] = None, inner_iters: Iterable[int] = (4, 6, 8, 12),
             wdepths: Iterable[int] = (None,), restarts: Iterable[int] = (None,),
             strip_rows: Iterable[int] = (None,), coarse_threads: Iterable[int] = (None,),
             per_iteration: bool = False, nus: Iterable[int] = (None,)):
    """Time one whole KKT solve (after ``fwi.forward``) per (inner-iteration
    count, W-cycle depth, FGMRES restart, column-strip height of the stencil
    kernels, threads per CTA of the shared-memory coarse cycle) and keep the
    fastest that converges (``nus``: Jacobi sweeps before and after each
    coarse-grid correction, nu1 = nu2).  With ``per_iteration`` the score is the time per
    FGMRES iteration: for launch-layout parameters, which change no arithmetic,
    the iteration count differs between candidates only through rounding (a
    few iterations either way) and would otherwise decide the choice.
    Returns (best Opts, table of (inner_iters, wdepth, restart, seconds, outer
    iterations, converged, strip_rows, coarse_threads, nu))."""
    import torch
    base = base if base is not None else default_opts()
    table = []
    best, best_t = None, math.inf
    for nu, n, wd, rs, sr, ct in itertools.product(nus, inner_iters, wdepths, restarts, strip_rows, coarse_threads):
        o = Opts.from_buffer_copy(base)
        o.inner_iters = n
        if nu is not None:
            o.nu1 = o.nu2 = nu
        if wd is not None:
            o.mg_wdepth = wd
        if rs is not None:
            o.restart = rs
        if sr is not None:
            o.strip_rows = sr
        if ct is not None:
            o.coarse_threads = ct
        if sr is not None:
            fwi.kkt_solve(o, allow_noconv=True)      # untimed: rebuilds the strip tables for this height
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ds, st = fwi.kkt_solve(o, allow_noconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = st["rel_res"] <= o.tol
        table.append((n, o.mg_wdepth, o.restart, dt, st["outer_iters"], ok, o.strip_rows, o.coarse_threads, o.nu1))
        score = dt / max(st["outer_iters"], 1) if per_iteration else dt
        if ok and score < best_t:
            best, best_t = o, score
    return (best if best is not None else base), table


def auto_wdepth(grids, freqs_per_grid, gammas, kh_max: float = 2.0, levels_max: int = 12) -> int:
    """Deepest multigrid level whose grid still resolves the wave field
    (omega h_l / c <= kh_max with c = 1/sqrt(mean gamma)), over every grid and
    frequency of a batch: the levels down to there repeat their coarse-grid
    correction (W), the coarser ones do not."""
    depth = 1
    for g, fr, gam in zip(grids, freqs_per_grid, gammas):
        c = 1.0 / math.sqrt(float(sum(map(float, [gam.mean()]))))
        for f in fr:
            om = 2.0 * math.pi * f
            l, h = 0, g.h
            while l + 1 < levels_max and om * (2.0 * h) / c <= kh_max:
                l += 1
                h *= 2.0
            depth = max(depth, l)
    return depth
