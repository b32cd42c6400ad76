"""Thin ctypes binding of ``include/fwikkt.h`` (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts numpy /
torch arguments to plain pointers and status codes to exceptions.  The
library is loaded from the in-tree build (``_lib/libfwikkt.so``); if it is
missing the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

from . import _build

FWI_OK = 0
FWI_E_INVAL = -1
FWI_E_NOMEM = -2
FWI_E_CUDA = -3
FWI_E_NOCONV = -4
FWI_E_NUMERIC = -5
FWI_C128 = 0
FWI_C64_REFINE = 1
FWI_DOT_RUNS = 0
FWI_DOT_FP64 = 1
FWI_DOT_COMP = 2
FWI_HBLOCK_MAX = 8

_ERRNAMES = {FWI_E_INVAL: "FWI_E_INVAL", FWI_E_NOMEM: "FWI_E_NOMEM", FWI_E_CUDA: "FWI_E_CUDA",
             FWI_E_NOCONV: "FWI_E_NOCONV", FWI_E_NUMERIC: "FWI_E_NUMERIC"}


class FwiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("npml", C.c_int), ("h", C.c_double),
                ("pml_c", C.c_double), ("pml_R", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eps", C.c_double), ("include_Ls_n", C.c_int),
                ("tol", C.c_double), ("restart", C.c_int), ("max_outer", C.c_int),
                ("sweep_tol", C.c_double), ("max_refine", C.c_int), ("inner_iters", C.c_int),
                ("inner_tol", C.c_double), ("mg_cycle", C.c_int), ("mg_wdepth", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("omega_jac", C.c_double), ("shift_beta", C.c_double), ("sigma_cap", C.c_double),
                ("mg_levels", C.c_int), ("fwd_tol", C.c_double), ("fwd_iters", C.c_int),
                ("max_fwd_refine", C.c_int), ("use_graph", C.c_int), ("arnoldi_dots", C.c_int),
                ("check_orth", C.c_int), ("strip_rows", C.c_int), ("coarse_threads", C.c_int),
                ("fwd_warm", C.c_int), ("outer_solver", C.c_int),
                ("inner_solver", C.c_int), ("hblock", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("refinements", C.c_int), ("fwd_sweeps", C.c_int),
                ("inner_iters", C.c_longlong), ("rel_res", C.c_double), ("misfit", C.c_double),
                ("t_setup_ms", C.c_double), ("t_forward_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("fwd_rel_res", C.c_double), ("orth_loss", C.c_double),
                ("fwd_warm", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LayoutInfo(C.Structure):
    _fields_ = [("n_instances", C.c_int), ("n_blocks", C.c_int), ("field_elems", C.c_longlong),
                ("ctrl_elems", C.c_longlong), ("kkt_elems", C.c_longlong)]


_lib = None
P = C.c_void_p
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int)


def header_functions() -> list:
    """Names of the functions declared in include/fwikkt.h."""
    txt = open(os.path.join(_build.INCLUDE, "fwikkt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z0-9_]+)\s*\(", txt)))


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the in-tree libfwikkt.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libfwikkt.so not built ({_build.LIB}); run paper_2204_06489_gb300._build.build()")
    L = C.CDLL(_build.LIB)
    sig = {
        "fwi_default_opts": (None, [C.POINTER(Opts)]),
        "fwi_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(Grid), P]),
        "fwi_set_survey": (C.c_int, [P, C.c_int, C.c_int, DP, C.c_int, IP, IP, DP, IP, IP, IP, DP]),
        "fwi_set_model": (C.c_int, [P, C.c_int, P, C.c_double, C.c_int]),
        "fwi_get_model": (C.c_int, [P, C.c_int, DP]),
        "fwi_set_observed": (C.c_int, [P, C.c_int, P, C.c_int]),
        "fwi_forward": (C.c_int, [P, C.POINTER(Opts), DP, DP, C.POINTER(Stats)]),
        "fwi_get_wavefields": (C.c_int, [P, P]),
        "fwi_gradient": (C.c_int, [P, C.POINTER(Opts), DP, P, C.c_int, C.POINTER(Stats)]),
        "fwi_kkt_solve": (C.c_int, [P, C.POINTER(Opts), P, C.c_int, C.POINTER(Stats)]),
        "fwi_newton_step": (C.c_int, [P, C.POINTER(Opts), P, C.c_int, C.POINTER(Stats)]),
        "fwi_rsgn_step": (C.c_int, [P, C.POINTER(Opts), P, C.c_int, C.POINTER(Stats)]),
        "fwi_normal_lambda_max": (C.c_int, [P, C.POINTER(Opts), C.c_int, DP, C.POINTER(Stats)]),
        "fwi_hessian_apply": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int, C.POINTER(Stats)]),
        "fwi_hblock_set": (C.c_int, [P, C.c_int, P, P, C.c_int]),
        "fwi_apply_helmholtz": (C.c_int, [P, P, P, C.c_int, C.c_int]),
        "fwi_apply_kkt": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int]),
        "fwi_apply_precond": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int]),
        "fwi_inner_solve": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int, C.c_int]),
        "fwi_mg_cycle": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int]),
        "fwi_mg_cycle_noalloc": (C.c_int, [P, C.POINTER(Opts), P, P, C.c_int]),
        "fwi_get_layout": (C.c_int, [P, C.POINTER(LayoutInfo)]),
        "fwi_last_error": (C.c_char_p, [P]),
        "fwi_kernel_launches": (C.c_ulonglong, []),
        "fwi_memory_calls": (C.c_ulonglong, []),
        "fwi_kernel_profile": (C.c_int, [P, C.c_int, C.c_char_p, C.c_longlong]),
        "fwi_stencil_timer": (C.c_int, [P, C.c_int, DP, DP, C.POINTER(C.c_longlong), DP]),
        "fwi_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_opts(**kw) -> Opts:
    o = Opts()
    load().fwi_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _dp(a: np.ndarray):
    return a.ctypes.data_as(DP)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(IP)


def _tensor_ptr(t) -> int:
    """Device pointer of a contiguous CUDA torch tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class FWI:
    """One library context: ``n`` independent instances on the current CUDA device."""

    def __init__(self, grids: Sequence, stream: Optional[int] = None):
        L = load()
        self._L = L
        garr = (Grid * len(grids))()
        for i, g in enumerate(grids):
            garr[i] = Grid(int(g.nx), int(g.nz), int(g.npml), float(g.h), float(g.pml_c), float(g.pml_R))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        h = P()
        rc = L.fwi_create(C.byref(h), len(grids), garr, P(stream))
        if rc != FWI_OK:
            raise FwiError(rc, L.fwi_last_error(None).decode())
        self._h = h
        self.grids = list(grids)
        self.surveys = [None] * len(grids)

    def close(self):
        if getattr(self, "_h", None):
            self._L.fwi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, allow_noconv: bool = False):
        if rc == FWI_OK or (allow_noconv and rc == FWI_E_NOCONV):
            return rc
        raise FwiError(rc, self._L.fwi_last_error(self._h).decode())

    # ------------------------------------------------------------------ set-up
    def set_survey(self, inst: int, sv):
        n = sv.n_src
        freqs = np.ascontiguousarray(sv.freqs_hz, dtype=np.float64)
        amp = np.ascontiguousarray(np.asarray(sv.src_amp, dtype=np.complex128).view(np.float64))
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (sv.src_ix, sv.src_iz, sv.rec_offsets,
                                                                  sv.rec_ix, sv.rec_iz)]
        w = np.ascontiguousarray(sv.rec_w, dtype=np.float64)
        self._check(self._L.fwi_set_survey(self._h, inst, len(freqs), _dp(freqs), n, _ip(arrs[0]),
                                           _ip(arrs[1]), _dp(amp), _ip(arrs[2]), _ip(arrs[3]),
                                           _ip(arrs[4]), _dp(w)))
        self.surveys[inst] = sv

    def set_model(self, inst: int, gamma_core, gamma_ref: float = 0.0):
        try:
            import torch
            if isinstance(gamma_core, torch.Tensor) and gamma_core.is_cuda:
                t = gamma_core.detach().to(torch.float64).contiguous()
                return self._check(self._L.fwi_set_model(self._h, inst, P(_tensor_ptr(t)), gamma_ref, 1))
        except ImportError:
            pass
        a = np.ascontiguousarray(np.asarray(gamma_core, dtype=np.float64))
        self._check(self._L.fwi_set_model(self._h, inst, a.ctypes.data_as(P), gamma_ref, 0))

    def get_model(self, inst: int) -> np.ndarray:
        g = self.grids[inst]
        out = np.zeros(g.nz * g.nx)
        self._check(self._L.fwi_get_model(self._h, inst, _dp(out)))
        return out.reshape(g.nz, g.nx)

    def set_observed(self, inst: int, d):
        try:
            import torch
            if isinstance(d, torch.Tensor) and d.is_cuda:
                t = d.detach().to(torch.complex128).contiguous()
                return self._check(self._L.fwi_set_observed(self._h, inst, P(_tensor_ptr(t)), 1))
        except ImportError:
            pass
        a = np.ascontiguousarray(np.asarray(d, dtype=np.complex128))
        self._check(self._L.fwi_set_observed(self._h, inst, a.ctypes.data_as(P), 0))

    def layout(self) -> dict:
        li = LayoutInfo()
        self._check(self._L.fwi_get_layout(self._h, C.byref(li)))
        return {k: getattr(li, k) for k, _ in li._fields_}

    # ------------------------------------------------------------------ solves
    def forward(self, opts: Optional[Opts] = None, want_data: bool = True):
        """Returns (d_pred per instance [n_freq, rec_total] complex, misfit per instance, stats)."""
        st = Stats()
        n_inst = len(self.grids)
        tot = sum(len(s.freqs_hz) * int(s.rec_offsets[-1]) for s in self.surveys)
        dp = np.zeros(2 * max(tot, 1)) if want_data else None
        mis = np.zeros(n_inst)
        self._check(self._L.fwi_forward(self._h, C.byref(opts) if opts else None,
                                        _dp(dp) if want_data else None, _dp(mis), C.byref(st)))
        out = None
        if want_data:
            z = dp[:2 * tot].view(np.complex128)
            out, o = [], 0
            for s in self.surveys:
                n = len(s.freqs_hz) * int(s.rec_offsets[-1])
                out.append(z[o:o + n].reshape(len(s.freqs_hz), -1).copy())
                o += n
        return out, mis, st.as_dict()

    def wavefields(self):
        import torch
        lay = self.layout()
        u = torch.zeros(lay["field_elems"], dtype=torch.complex128, device="cuda")
        self._check(self._L.fwi_get_wavefields(self._h, P(u.data_ptr())))
        return u

    def gradient(self, opts: Optional[Opts] = None, out=None):
        """(misfit per instance, gradient of all cores [Nc] FP64 (numpy, or the given CUDA tensor), stats)."""
        st = Stats()
        mis = np.zeros(len(self.grids))
        lay = self.layout()
        if out is not None:
            rc = self._L.fwi_gradient(self._h, C.byref(opts) if opts else None, _dp(mis),
                                      P(_tensor_ptr(out)), 1, C.byref(st))
            self._check(rc)
            return mis, out, st.as_dict()
        g = np.zeros(lay["ctrl_elems"])
        self._check(self._L.fwi_gradient(self._h, C.byref(opts) if opts else None, _dp(mis),
                                         g.ctypes.data_as(P), 0, C.byref(st)))
        return mis, g, st.as_dict()

    def kkt_solve(self, opts: Optional[Opts] = None, allow_noconv: bool = False):
        st = Stats()
        ds = np.zeros(self.layout()["ctrl_elems"])
        rc = self._L.fwi_kkt_solve(self._h, C.byref(opts) if opts else None, ds.ctypes.data_as(P), 0,
                                   C.byref(st))
        self._check(rc, allow_noconv)
        return ds, st.as_dict()

    def newton_step(self, opts: Optional[Opts] = None, allow_noconv: bool = False):
        st = Stats()
        ds = np.zeros(self.layout()["ctrl_elems"])
        rc = self._L.fwi_newton_step(self._h, C.byref(opts) if opts else None, ds.ctypes.data_as(P), 0,
                                     C.byref(st))
        self._check(rc, allow_noconv)
        return ds, st.as_dict()

    def rsgn_step(self, opts: Optional[Opts] = None, allow_noconv: bool = False):
        """One reduced-space Gauss-Newton step (normal equations by CG); same
        outputs as ``newton_step`` (stats["outer_iters"] counts CG iterations)."""
        st = Stats()
        ds = np.zeros(self.layout()["ctrl_elems"])
        rc = self._L.fwi_rsgn_step(self._h, C.byref(opts) if opts else None, ds.ctypes.data_as(P), 0,
                                   C.byref(st))
        self._check(rc, allow_noconv)
        return ds, st.as_dict()

    def normal_lambda_max(self, opts: Optional[Opts] = None, iters: int = 10):
        """Power-iteration estimate of the largest eigenvalue of the Gauss-Newton
        matrix Re(J~^H W^T W J~) at the current models (needs ``forward``)."""
        st = Stats()
        lam = C.c_double()
        rc = self._L.fwi_normal_lambda_max(self._h, C.byref(opts) if opts else None, int(iters), C.byref(lam),
                                           C.byref(st))
        self._check(rc)
        return lam.value, st.as_dict()

    def hessian_apply(self, v, opts: Optional[Opts] = None, allow_noconv: bool = False):
        """H~ v of the reduced Gauss-Newton system at the current models, in the
        scaled control (ds / gamma_ref); ``v`` a numpy array (returns numpy) or
        a CUDA float64 tensor (returns a tensor).  Needs ``forward``."""
        st = Stats()
        o = C.byref(opts) if opts else None
        if isinstance(v, np.ndarray):
            vv = np.ascontiguousarray(v, dtype=np.float64)
            out = np.empty_like(vv)
            rc = self._L.fwi_hessian_apply(self._h, o, vv.ctypes.data, out.ctypes.data, 0, C.byref(st))
        else:
            vv = v.contiguous()
            out = vv.new_empty(vv.shape)
            rc = self._L.fwi_hessian_apply(self._h, o, _tensor_ptr(vv), _tensor_ptr(out), 1, C.byref(st))
        self._check(rc, allow_noconv)
        return out, st.as_dict()

    def hblock_set(self, S=None, Y=None):
        """Curvature pairs (rows of S, Y, scaled control, oldest first) of the
        quasi-Newton H block (opts.hblock = 1); no arguments removes them."""
        if S is None:
            self._check(self._L.fwi_hblock_set(self._h, 0, None, None, 0))
            return
        if isinstance(S, np.ndarray):
            Sa = np.ascontiguousarray(S, dtype=np.float64)
            Ya = np.ascontiguousarray(Y, dtype=np.float64)
            if Sa.shape != Ya.shape or Sa.ndim != 2:
                raise ValueError("S and Y must be [m, ctrl_elems]")
            self._check(self._L.fwi_hblock_set(self._h, Sa.shape[0], Sa.ctypes.data, Ya.ctypes.data, 0))
        else:
            Sa, Ya = S.contiguous(), Y.contiguous()
            if Sa.shape != Ya.shape or Sa.dim() != 2:
                raise ValueError("S and Y must be [m, ctrl_elems]")
            self._check(self._L.fwi_hblock_set(self._h, Sa.shape[0], _tensor_ptr(Sa), _tensor_ptr(Ya), 1))

    def kernel_profile(self, enable: int):
        """The library's kernel profile since the last reset (a dict with
        gap_ms, gaps and rows of kernel, level, launches, ms, bytes); ``enable``
        1/0 then clears it and switches it on/off, -1 only reads."""
        import json
        n = 1 << 16
        while True:
            buf = C.create_string_buffer(n)
            rc = self._L.fwi_kernel_profile(self._h, -1, buf, n)
            if rc == FWI_OK:
                break
            if n > (1 << 26):
                self._check(rc)
            n *= 4
        self._check(self._L.fwi_kernel_profile(self._h, enable, None, 0))
        return json.loads(buf.value.decode())

    def stencil_timer(self, enable: int, with_pass: bool = False):
        """(ms, algorithmic bytes, launches[, fused-pass bytes]) of the level-0
        two-sweep smoother kernel since the last reset; ``enable`` 1/0 resets
        and switches timing, -1 reads."""
        ms, by, n, pb = C.c_double(), C.c_double(), C.c_longlong(), C.c_double()
        self._check(self._L.fwi_stencil_timer(self._h, enable, C.byref(ms), C.byref(by), C.byref(n), C.byref(pb)))
        if with_pass:
            return ms.value, by.value, n.value, pb.value
        return ms.value, by.value, n.value

    # ------------------------------------------------------------------ operators (torch CUDA tensors)
    @staticmethod
    def _prec_of(t) -> int:
        import torch
        if t.dtype in (torch.complex128, torch.float64):
            return FWI_C128
        if t.dtype in (torch.complex64, torch.float32):
            return FWI_C64_REFINE
        raise TypeError(f"unsupported dtype {t.dtype}")

    def apply_helmholtz(self, x, adjoint: bool = False):
        import torch
        y = torch.empty_like(x)
        self._check(self._L.fwi_apply_helmholtz(self._h, P(_tensor_ptr(x)), P(_tensor_ptr(y)),
                                                int(adjoint), self._prec_of(x)))
        return y

    def apply_kkt(self, xi, opts: Optional[Opts] = None):
        import torch
        y = torch.empty_like(xi)
        self._check(self._L.fwi_apply_kkt(self._h, C.byref(opts) if opts else None, P(_tensor_ptr(xi)),
                                          P(_tensor_ptr(y)), self._prec_of(xi)))
        return y

    def apply_precond(self, v, opts: Optional[Opts] = None):
        import torch
        z = torch.empty_like(v)
        self._check(self._L.fwi_apply_precond(self._h, C.byref(opts) if opts else None, P(_tensor_ptr(v)),
                                              P(_tensor_ptr(z)), self._prec_of(v)))
        return z

    def inner_solve(self, b, opts: Optional[Opts] = None, adjoint: bool = False):
        import torch
        x = torch.empty_like(b)
        self._check(self._L.fwi_inner_solve(self._h, C.byref(opts) if opts else None, P(_tensor_ptr(b)),
                                            P(_tensor_ptr(x)), int(adjoint), self._prec_of(b)))
        return x

    def mg_cycle(self, b, opts: Optional[Opts] = None):
        import torch
        x = torch.empty_like(b)
        self._check(self._L.fwi_mg_cycle(self._h, C.byref(opts) if opts else None, P(_tensor_ptr(b)),
                                         P(_tensor_ptr(x)), self._prec_of(b)))
        return x


def from_workload(workloads, stream=None) -> FWI:
    """Context for one or more :class:`fwi_inputs.Workload` at their starting models."""
    if not isinstance(workloads, (list, tuple)):
        workloads = [workloads]
    f = FWI([w.grid for w in workloads], stream)
    for i, w in enumerate(workloads):
        f.set_survey(i, w.survey)
        f.set_model(i, w.gamma_start)
    return f
