"""GB300-native full-space Gauss-Newton FWI (Malovichko, Orazbayev & Khokhlov).

The hot path -- the preconditioned Krylov solve of each Newton step's KKT
system (Sec. 4-5) -- runs in the CUDA library ``libfwikkt.so`` behind the C
ABI of ``include/fwikkt.h``; :mod:`.api` is its thin ctypes binding and
:mod:`.autograd` wraps the misfit and its adjoint gradient as a
``torch.autograd.Function``.
"""
from .api import (FWI, FwiError, Opts, default_opts, from_workload, load, lib_path,  # noqa: F401
                  FWI_C128, FWI_C64_REFINE, FWI_OK, FWI_E_INVAL, FWI_E_NOMEM, FWI_E_CUDA,
                  FWI_E_NOCONV, FWI_E_NUMERIC)
