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


@pytest.mark.parametrize("case", ["density_current", "hill", "squall"])
def test_warp_per_column_solves_match_the_thread_per_column_ones(case):
    """ERF_OPT_WARP_COLUMNS: the FP64 column kernels with one warp per column (the system built by
    the lanes at once, the substitutions as a warp scan of segment maps) against one thread per
    column: 4 steps agree to 1e-13 relative L2 (rounding of the segment joins only; dry slab,
    terrain, moist).  Grids below 2^15 columns run the warp form by default, so every smaller
    parity test also holds it to the oracle's 1e-11."""
    from paper_2412_04395_gb300 import workloads as W
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_WARP_COLUMNS
    if case == "density_current":
        wl = W.density_current(nx=72, ny=3, nz=40, dx=300.0)
    elif case == "hill":
        wl = W.hill_bubble(nx=40, ny=36, nz=30, dx=200.0, dz0=60.0, ratio=1.03, h0=300.0)
    else:
        wl = W.squall_line(nx=64, ny=3, nz=48, dx=500.0, dt=2.0, relax_width=5000.0)
    out = []
    for mode in (0, 1):
        d = Dycore(wl)
        if wl.moist:
            d.erf_set_initial_moist(wl.dtheta, wl.qv, wl.u, wl.v, wl.w)
        else:
            d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
        d.erf_set_option(ERF_OPT_WARP_COLUMNS, mode)
        assert d.erf_get_option(ERF_OPT_WARP_COLUMNS) == mode
        d.erf_rk3_step(4)
        out.append(d.state())
        d.close()
    mom = np.sqrt(sum(np.linalg.norm(out[0][f]) ** 2 for f in ("rhou", "rhov", "rhow")))
    for f in out[0]:
        den = mom if f in ("rhou", "rhov", "rhow") else np.linalg.norm(out[0][f])
        assert np.linalg.norm(out[0][f] - out[1][f]) <= 1e-13 * den, (case, f)
