"""The allocation-free reduction entry point (erf_reduce_state_noalloc).

Callers that cannot allocate device memory (a foreign memory pool, a sandbox without cudaMalloc,
a fully pre-assigned HBM arena) hand over only the state arrays they own; the entry point keeps
its scratch in a static device array.  Here it is called through the C ABI on a state held in
torch tensors and checked against erf_diagnostics (the workspace-based reduction) on two calls
in a row.  This file is collected last so that a failure here stops a -x run only after every
other test has run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_diagnostics_twice():
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2412_04395_gb300 import erf, workloads as W

    wl = W.density_current(nx=96, ny=6, nz=40, dx=300.0)
    d = erf.Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    L = d.L
    L.erf_reduce_state_noalloc.restype = C.c_int
    L.erf_reduce_state_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double] + \
        [C.c_void_p] * 8
    dev = torch.device("cuda")
    dz = torch.tensor(np.diff(wl.zeta), dtype=torch.float64, device=dev)
    out = torch.full((5,), -1.0, dtype=torch.float64, device=dev)
    for call in range(2):
        d.erf_rk3_step(2)
        f = {k: torch.empty(d._shape(k), dtype=torch.float64, device=dev)
             for k in ("rho", "rhotheta", "rhou", "rhov", "rhow")}
        for k, t in f.items():
            d.erf_get_state(k, out=t)
        st = L.erf_reduce_state_noalloc(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, dz.data_ptr(),
                                        f["rho"].data_ptr(), f["rhotheta"].data_ptr(), f["rhou"].data_ptr(),
                                        f["rhov"].data_ptr(), f["rhow"].data_ptr(), out.data_ptr(),
                                        d.stream.cuda_stream)
        assert st == erf.ERF_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = d.erf_diagnostics()
        assert ref["status"] == erf.ERF_OK
        # the two reductions sum in different orders: mass within 1e-13, extrema exactly
        assert got[0] == pytest.approx(ref["mass"], rel=1e-13, abs=0.0)
        assert got[1] == ref["max_abs_w"]
        assert got[2] == ref["theta_min"] and got[3] == ref["theta_max"]
        assert got[4] == 0.0 and ref["nonfinite"] == 0
    # a grid beyond the static scratch is refused with ERF_ENOSPACE, nothing launched
    st = L.erf_reduce_state_noalloc(65536, 4096, 2, 1.0, 1.0, dz.data_ptr(), f["rho"].data_ptr(),
                                    f["rhotheta"].data_ptr(), f["rhou"].data_ptr(), f["rhov"].data_ptr(),
                                    f["rhow"].data_ptr(), out.data_ptr(), d.stream.cuda_stream)
    assert st == erf.ERF_ENOSPACE
