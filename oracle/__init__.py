"""CPU oracle for full-space Gauss-Newton FWI (Malovichko, Orazbayev & Khokhlov).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, double-precision
(complex128) restatement of the discretised problem of the paper: the PML
Helmholtz operator (Sec. 2, eq. helmholtz_preliminary), the observation
operator (Sec. 2), the reduced Gauss-Newton system (Sec. 3), the KKT system
(Sec. 4, eq. KKT), the block-triangular preconditioners (Sec. 5, eqs. precond
and precond_approx) and GMRES on the KKT matrix.  It uses scipy sparse LU for the
Helmholtz blocks.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the CUDA library shares no code with
it (the two meet only in :mod:`fwi_inputs`, which describes problems and holds no
arithmetic of the method).

Modules
-------
grid       padded grid, PML stretching functions, model embedding
helmholtz  sparse operator assembly, sources, receivers
fwi        forward modelling, data residual, misfit, adjoint gradient
kkt        scaled KKT matvec / RHS, exact and inexact preconditioners, direct
           references (real-form sparse KKT, dense normal equations), the
           matrix-free normal operator of RSGN-CG (Sec. 3)
krylov     flexible GMRES in the real inner product, BiCGStab, CG
mg         geometric multigrid for the shifted operator (the inner block solver)
ilu        ILU(0) of the 5-point operator (the paper's incomplete-LU block approximation)
lbfgs      L-BFGS inverse of the reduced Hessian for the preconditioner's H block

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a library routine, an invariant or brute force.  The multigrid
cycle (the paper leaves the inner solver open; Sec. 5 names only "shifted
Laplacian with multigrid") is pinned by exact Fourier analysis: on grids
without the layer, with constant gamma and 2^k - 1 nodes per side, the cycle
applied to every sine mode equals its closed-form two-, three- and four-grid
symbol (damped Jacobi, full weighting, bilinear interpolation, rediscretised
coarse operators, V/W recursion); the coarse levels' layer profile is pinned
by the positions of the coarse nodes on the fine profile.  The inner BiCGStab
is pinned iterate by iterate against scipy.sparse.linalg.bicgstab, the
coupling block P~ by finite differences of the forward data.
"""
