"""fwi_mg_cycle_noalloc: the multigrid cycle for callers that cannot allocate
device memory during the call (their memory belongs to another pool, or they
run next to busy streams where cudaMalloc/cudaFree would block).  Its level
buffers live in a static device array of the library, so it must give the
same result as fwi_mg_cycle, call after call, and make no cudaMalloc /
cudaFree (the library's own count of memory calls and the device's free
memory stay unchanged, with the live stencil timer switched on).  Collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

import fwi_inputs as FI

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(P, wls):
    f = P.from_workload(wls)
    return f


def _run(f, fn, opts, b):
    x = torch.empty_like(b)
    prec = f._prec_of(b)
    rc = fn(f._h, C.byref(opts), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), prec)
    f._check(rc)
    torch.cuda.synchronize()
    return x


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-10), (torch.complex64, 2e-5)])
def test_noalloc_cycle_matches_allocating_cycle(lib, dtype, tol):
    import paper_2204_06489_gb300 as P
    wl_a = FI.tiny_workload(seed=0)
    wl_b = FI.micro_workload(seed=1, nx=37, nz=23, npml=6, n_src=3, n_rec=5)
    f = _ctx(P, [wl_a, wl_b])
    opts = P.default_opts()
    n = f.layout()["field_elems"]
    g = np.random.default_rng(21)
    b = torch.from_numpy(g.standard_normal(n) + 1j * g.standard_normal(n)).to(dtype).cuda()
    ref = _run(f, lib.fwi_mg_cycle, opts, b)            # builds the hierarchy (allocating call)
    x = torch.empty_like(b)
    prec = f._prec_of(b)

    def call():
        f._check(lib.fwi_mg_cycle_noalloc(f._h, C.byref(opts), C.c_void_p(b.data_ptr()),
                                          C.c_void_p(x.data_ptr()), prec))
        torch.cuda.synchronize()

    call()                                              # first call: loads the kernels, looks up the array
    # the live stencil timer allocates its event buffers on first use; inside
    # this call it must stay off, so the call still allocates nothing
    f.stencil_timer(1)
    outs = [torch.empty_like(b) for _ in range(2)]
    torch.linalg.vector_norm(outs[0] - ref)             # torch reserves its own memory before the check
    torch.cuda.synchronize()
    # only the two library calls (and device-to-device copies into buffers
    # that already exist) run between the two readings of free device memory
    free0, _ = torch.cuda.mem_get_info()
    calls0 = lib.fwi_memory_calls()
    for k in range(2):                                  # two calls in a row share the static array
        call()
        outs[k].copy_(x)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert lib.fwi_memory_calls() == calls0
    assert free1 == free0, (free0, free1)
    for out in outs:
        rel = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert rel < tol, rel
    f.stencil_timer(0)
    f.close()


def test_noalloc_cycle_rejects_oversized_batch_and_missing_setup(lib):
    import paper_2204_06489_gb300 as P
    wl = FI.marmousi_shaped_workload(n_src=16, freqs=(5.0,))
    f = _ctx(P, wl)
    opts = P.default_opts()
    n = f.layout()["field_elems"]
    b = torch.zeros(n, dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    # no hierarchy yet: refused, nothing allocated on its behalf
    rc = lib.fwi_mg_cycle_noalloc(f._h, C.byref(opts), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                  P.FWI_C128)
    assert rc == P.FWI_E_INVAL
    _run(f, lib.fwi_mg_cycle, opts, b)
    rc = lib.fwi_mg_cycle_noalloc(f._h, C.byref(opts), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                  P.FWI_C128)
    assert rc == P.FWI_E_INVAL
    assert b"FWI_NOALLOC_SCRATCH_BYTES" in lib.fwi_last_error(f._h)
    f.close()
