"""Mixed-precision substep (App. C rows 3-5): the explicit vertical part run inside the column
sweep of the tridiagonal solve (one thread per column) must give results bit for bit equal to
the per-cell kernel followed by the sweep, with and without the passive scalar's flux sums, on
even and ragged grids (nx % 4 != 0 takes the scalar finishing kernel)."""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def _run(wl, fused, steps):
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_COLUMN_FUSION
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if getattr(wl, "tracer", 0):
        d.erf_set_tracer_initial(wl.phi)
    d.erf_set_option(ERF_OPT_COLUMN_FUSION, fused)
    assert d.erf_get_option(ERF_OPT_COLUMN_FUSION) == fused
    d.erf_rk3_step(steps)
    assert d.erf_diagnostics()["status"] == 0
    st = d.state()
    if getattr(wl, "tracer", 0):
        st["rhophi"] = d.erf_get_state("rhophi")
    return st


@pytest.mark.parametrize("shape,tracer", [((64, 48, 40), False), ((30, 28, 40), True), ((64, 16, 24), True)])
def test_fused_column_sweep_matches_split_kernels(shape, tracer):
    nx, ny, nz = shape
    wl = W.convective_abl(nx=nx, ny=ny, nz=nz, dx=40.0)
    if tracer:
        wl = W.with_tracer(wl, "blob", radius_frac=0.3)
    a = _run(wl, 1, 4)
    b = _run(wl, 0, 4)
    for f in a:
        assert np.array_equal(a[f], b[f]), f


def test_column_fusion_default_follows_the_column_count():
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_COLUMN_FUSION
    small = W.convective_abl(nx=64, ny=64, nz=16, dx=40.0)
    d = Dycore(small)
    assert d.erf_get_option(ERF_OPT_COLUMN_FUSION) == 0
    d.erf_set_option(ERF_OPT_COLUMN_FUSION, -1)
    assert d.erf_get_option(ERF_OPT_COLUMN_FUSION) == 0
