"""TMA-staged stencils (mixed path): the shared-memory tile kernel must give results bit for bit
equal to the plain-load kernel, on grids whose tiles fit exactly and on ragged ones (nx not a
multiple of the tile width, ny and nz not multiples of the tile height), with the periodic halo
patched at every domain edge."""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


@pytest.mark.parametrize("shape", [(128, 64, 32), (100, 18, 22)])
def test_tma_tiles_match_plain_loads(shape):
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_TMA_STENCILS
    nx, ny, nz = shape
    wl = W.convective_abl(nx=nx, ny=ny, nz=nz, dx=40.0)
    a = Dycore(wl)
    a.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    b = Dycore(wl)
    b.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    b.erf_set_option(ERF_OPT_TMA_STENCILS, 0)
    assert a.erf_get_option(ERF_OPT_TMA_STENCILS) == 1
    assert b.erf_get_option(ERF_OPT_TMA_STENCILS) == 0
    a.erf_rk3_step(5)
    b.erf_rk3_step(5)
    assert a.erf_diagnostics()["status"] == 0
    sa, sb = a.state(), b.state()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f


def test_tma_not_used_where_the_grid_does_not_allow_it():
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_TMA_STENCILS
    wl = W.convective_abl(nx=30, ny=28, nz=40, dx=40.0)   # nx % 4 != 0
    d = Dycore(wl)
    assert d.erf_get_option(ERF_OPT_TMA_STENCILS) == 0


def test_bounded_wait_gives_up_and_reports():
    """An mbarrier armed for bytes that never arrive: the kernel's wait gives up after its poll
    limit, sets the error word and returns; the context stays usable for a normal step."""
    from paper_2412_04395_gb300 import erf
    from paper_2412_04395_gb300.erf import Dycore
    assert erf.erf_selftest_wait_timeout(1000) == 1
    wl = W.convective_abl(nx=64, ny=16, nz=16, dx=40.0)
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    d.erf_rk3_step(1)
    assert d.erf_diagnostics()["status"] == 0
