"""The C ABI library builds, loads and exports every function declared in
include/fwikkt.h; host-only calls validate their arguments.  CPU only (no
compute calls)."""
import ctypes as C

import numpy as np
import pytest

import fwi_inputs as FI


@pytest.fixture(scope="module")
def L():
    from paper_2204_06489_gb300 import _build, api
    _build.build()
    return api.load()


def test_every_declared_function_is_exported(L):
    from paper_2204_06489_gb300 import api
    names = api.header_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_default_opts(L):
    from paper_2204_06489_gb300 import api
    o = api.default_opts()
    assert o.restart == 30 and o.tol == 1e-6 and o.precision == api.FWI_C64_REFINE
    assert o.mg_cycle == 2 and o.nu1 == 2 and o.shift_beta == 0.5


def test_create_rejects_bad_grids_and_survey(L):
    from paper_2204_06489_gb300 import api
    bad = (api.Grid * 1)(api.Grid(1, 10, 4, 10.0, 3000.0, 1e-3))
    h = C.c_void_p()
    assert L.fwi_create(C.byref(h), 1, bad, None) == api.FWI_E_INVAL
    assert b"invalid grid" in L.fwi_last_error(None)
    good = (api.Grid * 1)(api.Grid(11, 9, 3, 10.0, 3000.0, 1e-3))
    assert L.fwi_create(C.byref(h), 1, good, None) == api.FWI_OK
    f = np.array([5.0])
    sx = np.array([20], dtype=np.int32)   # outside the 11-node core
    sz = np.array([2], dtype=np.int32)
    amp = np.array([1.0, 0.0])
    ro = np.array([0, 1], dtype=np.int32)
    rx = np.array([3], dtype=np.int32)
    rz = np.array([2], dtype=np.int32)
    dp = lambda a: a.ctypes.data_as(api.DP)
    ip = lambda a: a.ctypes.data_as(api.IP)
    rc = L.fwi_set_survey(h, 0, 1, dp(f), 1, ip(sx), ip(sz), dp(amp), ip(ro), ip(rx), ip(rz), None)
    assert rc == api.FWI_E_INVAL and b"source outside" in L.fwi_last_error(h)
    sx[0] = 5
    rc = L.fwi_set_survey(h, 0, 1, dp(f), 1, ip(sx), ip(sz), dp(amp), ip(ro), ip(rx), ip(rz), None)
    assert rc == api.FWI_OK
    assert L.fwi_set_survey(h, 3, 1, dp(f), 1, ip(sx), ip(sz), dp(amp), ip(ro), ip(rx), ip(rz), None) == api.FWI_E_INVAL
    L.fwi_destroy(h)
    L.fwi_destroy(None)


def test_solver_entry_points_reject_a_null_context(L):
    """Host-side argument check of the stepping and solving calls: a NULL
    context is FWI_E_INVAL before any device work."""
    from paper_2204_06489_gb300 import api
    st = api.Stats()
    ds = np.zeros(4)
    o = api.default_opts()
    for name in ("fwi_newton_step", "fwi_rsgn_step", "fwi_kkt_solve"):
        fn = getattr(L, name)
        assert fn(None, C.byref(o), ds.ctypes.data_as(api.DP), 0, C.byref(st)) == api.FWI_E_INVAL, name


def test_product_path_has_no_cpu_fallback():
    """The binding loads only the in-tree CUDA library and never imports the oracle."""
    import importlib
    import sys
    for m in [k for k in sys.modules if k.startswith("paper_2204_06489_gb300")]:
        del sys.modules[m]
    before = set(k for k in sys.modules if k.startswith("oracle"))
    importlib.import_module("paper_2204_06489_gb300")
    after = set(k for k in sys.modules if k.startswith("oracle"))
    assert after == before
    src = open(__import__("paper_2204_06489_gb300.api", fromlist=["x"]).__file__).read()
    assert "import oracle" not in src and "from oracle" not in src

