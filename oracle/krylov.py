"""Krylov solvers of the oracle: flexible GMRES and BiCGStab.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 5: the preconditioned KKT matrix is non-symmetric, so GMRES is used
(FSGN-GMRes); Sec. 6 fixes 30 GMRES iterations per cycle.  With an inexact
preconditioner that is itself an iterative solve (eq. precond_approx with a
Krylov inner solver) the preconditioner changes from one application to the
next, so the right-preconditioned *flexible* form (Saad 1993) is used; with a
fixed linear preconditioner it reduces to right-preconditioned GMRES.  The
inner product is the real one, <x, y> = x . y on the packed real vector.

Conjugate gradients (Hestenes & Stiefel 1952) solve the reduced-space normal
equations of Sec. 3 (RSGN-CG), whose matrix is symmetric positive definite for
eps > 0.

BiCGStab (van der Vorst 1992) with right preconditioning is the inner block
solver of the inexact preconditioner; Sec. 7 mentions BiCGStab as a
memory-lean alternative.  It works on complex vectors with the Hermitian inner
product <a, b> = sum conj(a) b.
"""
from __future__ import annotations

import numpy as np


def fgmres(matvec, b: np.ndarray, precond=None, restart: int = 30, tol: float = 1e-6,
           max_iter: int = 300, x0: np.ndarray | None = None):
    """Right-preconditioned flexible GMRES(restart), modified Gram-Schmidt,
    Givens rotations; stops when the true relative residual ||b - M x|| / ||b||
    (recomputed at the end of every cycle) is <= tol.

    Returns (x, info) with info = dict(iters, true_relres, history) where history
    lists the Givens residual estimates relative to ||b||."""
    if precond is None:
        def precond(v):
            return v
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    info = dict(iters=0, true_relres=0.0, history=[], cycles=0)
    if bnorm == 0.0:
        return x, info
    r = b - matvec(x) if x0 is not None else b.copy()
    beta = float(np.linalg.norm(r))
    while info["iters"] < max_iter:
        if beta / bnorm <= tol:
            break
        m = restart
        V = np.zeros((m + 1, n))
        Zs = np.zeros((m, n))
        Hh = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Zs[j] = precond(V[j])
            w = matvec(Zs[j])
            for i in range(j + 1):
                Hh[i, j] = float(np.dot(w, V[i]))
                w = w - Hh[i, j] * V[i]
            Hh[j + 1, j] = float(np.linalg.norm(w))
            if Hh[j + 1, j] > 0.0:
                V[j + 1] = w / Hh[j + 1, j]
            for i in range(j):                     # previous rotations
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            rr = np.hypot(Hh[j, j], Hh[j + 1, j])
            cs[j] = Hh[j, j] / rr
            sn[j] = Hh[j + 1, j] / rr
            Hh[j, j] = rr
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info["iters"] += 1
            info["history"].append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or info["iters"] >= max_iter:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):             # back substitution
            y[i] = (g[i] - np.dot(Hh[i, i + 1:k], y[i + 1:k])) / Hh[i, i]
        x = x + Zs[:k].T @ y
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        info["cycles"] += 1
    info["true_relres"] = beta / bnorm
    return x, info


def bicgstab(apply_A, b: np.ndarray, precond=None, iters: int = 10, tol: float = 0.0):
    """Right-preconditioned BiCGStab from x0 = 0, shadow residual r^ = b.

    Runs ``iters`` iterations (or stops early when ||r|| <= tol ||b||).  Guards:
    a vanishing denominator ends the iteration with the current x.
    Returns (x, relres_history)."""
    if precond is None:
        def precond(v):
            return v
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    bn = np.linalg.norm(b)
    hist = []
    if bn == 0.0:
        return x, hist
    rho_old = alpha = om = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(iters):
        rho = np.vdot(rh, r)
        if rho == 0.0:
            break
        beta = (rho / rho_old) * (alpha / om)
        p = r + beta * (p - om * v)
        ph = precond(p)
        v = apply_A(ph)
        den = np.vdot(rh, v)
        if den == 0.0:
            break
        alpha = rho / den
        s = r - alpha * v
        sh = precond(s)
        t = apply_A(sh)
        tt = np.vdot(t, t).real
        om = np.vdot(t, s) / tt if tt > 0.0 else 0.0
        x = x + alpha * ph + om * sh
        r = s - om * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / bn)
        if tol > 0.0 and hist[-1] <= tol:
            break
        if om == 0.0:
            break
    return x, hist


def cg(apply_H, g: np.ndarray, tol: float = 1e-6, max_iter: int = 1000):
    """Unpreconditioned conjugate gradients for H x = g, H symmetric positive
    definite (real vectors), from x = 0, stopping when the recursively updated
    residual satisfies ||r|| <= tol ||g||.  Returns (x, relres_history)."""
    x = np.zeros_like(g)
    r = g.copy()
    p = r.copy()
    gn = np.linalg.norm(g)
    hist = []
    if gn == 0.0:
        return x, hist
    rho = float(r @ r)
    for _ in range(max_iter):
        hp = apply_H(p)
        alpha = rho / float(p @ hp)
        x = x + alpha * p
        r = r - alpha * hp
        rho_new = float(r @ r)
        hist.append(np.sqrt(rho_new) / gn)
        if hist[-1] <= tol:
            break
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, hist
