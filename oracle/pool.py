"""Exact block solves of the oracle spread over a pool of host processes.

TEST INFRASTRUCTURE ONLY (see the package docstring): used to time the oracle
on the host cores (the CPU baseline of the benchmark).  It adds no arithmetic
of the method: every worker runs ``fwi.solve`` (sparse LU of A'_f, factorised
once per worker and frequency on first use) on a contiguous range of the
(frequency, source) blocks, which are independent (Sec. 2, one Helmholtz
problem per source and frequency).  Right-hand sides and solutions travel
through two shared-memory [B, N] complex128 arrays.  Workers are started with
the ``spawn`` method and with one BLAS thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import fwi

_W = {}


def _init(grid, survey, gamma_pad_fixed, gamma_ref, s_core, shape, names):
    prob = fwi.Problem(grid, survey, gamma_pad_fixed, gamma_ref)
    shms = [shared_memory.SharedMemory(name=n) for n in names]
    arrs = [np.ndarray(shape, dtype=np.complex128, buffer=m.buf) for m in shms]
    _W.update(prob=prob, s=np.asarray(s_core, dtype=np.float64), shms=shms, rhs=arrs[0], out=arrs[1])


def _solve_range(args):
    b0, b1, adjoint = args
    prob, s = _W["prob"], _W["s"]
    for b in range(b0, b1):
        _W["out"][b] = fwi.solve(prob, s, prob.block_freq(b), _W["rhs"][b], adjoint)
    return b1 - b0


class BlockPool:
    """``solve(rhs [B, N], adjoint) -> [B, N]``: A'^{-1} (or A'^{-H}) of every
    block at the model ``s_core``, by ``workers`` processes."""

    def __init__(self, prob: fwi.Problem, s_core, workers: int):
        Nz, Nx = prob.grid.nz + 2 * prob.grid.npml, prob.grid.nx + 2 * prob.grid.npml
        self.shape = (prob.n_blocks, Nz * Nx)
        nbytes = int(np.prod(self.shape)) * 16
        self.shms = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(2)]
        self.rhs = np.ndarray(self.shape, dtype=np.complex128, buffer=self.shms[0].buf)
        self.out = np.ndarray(self.shape, dtype=np.complex128, buffer=self.shms[1].buf)
        self.workers = int(workers)
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            ctx = mp.get_context("spawn")
            self.pool = ctx.Pool(self.workers, initializer=_init,
                                 initargs=(prob.grid, prob.survey, prob.gamma_pad_fixed, prob.gamma_ref,
                                           np.asarray(s_core), self.shape, [m.name for m in self.shms]))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        B = self.shape[0]
        step = -(-B // self.workers)
        self.ranges = [(b0, min(B, b0 + step)) for b0 in range(0, B, step)]

    def warm(self):
        """Start the workers (interpreter start-up only; nothing factorised)."""
        self.pool.map(int, range(self.workers))

    def solve(self, rhs: np.ndarray, adjoint: bool) -> np.ndarray:
        self.rhs[...] = rhs
        self.pool.map(_solve_range, [(b0, b1, adjoint) for b0, b1 in self.ranges])
        return self.out.copy()

    def close(self):
        self.pool.terminate()
        self.pool.join()
        for m in self.shms:
            m.close()
            m.unlink()
