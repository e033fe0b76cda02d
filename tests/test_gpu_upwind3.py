"""Third-order upwind advection (Sec. 3.6; the paper's scaling workload of Sec. 5.2 uses it for
momenta and scalars) on the GPU against the FP64 oracle through the C ABI: FP64 within 1e-11
relative L2 per field at the configured density-current steps and on small windows of the
scaling workload and of the hill bubble; the mixed-precision path within its FP32 bounds; TMA
tiles bit-identical to plain loads with the upwind-3 interpolant."""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

pytestmark = pytest.mark.gpu
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def _gpu(wl):
    from paper_2412_04395_gb300.erf import Dycore
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    return d


def _errs(g, r, per_field):
    """rho, rho theta and (per_field) every non-zero momentum against its own norm; otherwise
    momenta against the momentum-vector norm."""
    mom = np.sqrt(sum(np.linalg.norm(r[f]) ** 2 for f in ("rhou", "rhov", "rhow")))
    out = {}
    for f in FIELDS:
        own = np.linalg.norm(r[f])
        den = own if (f in ("rho", "rhotheta") or (per_field and own > 1e-14 * mom)) else mom
        out[f] = float(np.linalg.norm(g[f] - r[f]) / den)
    return out


def _u3(wl):
    return wl.with_(mom_adv=W.MOM_UPWIND3, scal_adv=W.SCAL_UPWIND3)


def test_fp64_upwind3_density_current_configured_steps():
    wl = _u3(W.density_current())
    o = make_oracle(wl)
    d = _gpu(wl)
    o.step(wl.steps)
    d.erf_rk3_step(wl.steps)
    e = _errs(d.state(), o.state(), per_field=True)
    print("upwind-3 density current 100 steps:", e)
    assert all(v <= 1e-11 for v in e.values()), e


@pytest.mark.parametrize("case", ["paper_scaling", "hill"])
def test_fp64_upwind3_windows(case):
    if case == "paper_scaling":
        wl = W.paper_scaling(nx=40, ny=36, nz=48)
        steps = 20
    else:
        wl = _u3(W.hill_bubble(nx=32, ny=40, nz=64, dx=100.0))
        steps = 40
    o = make_oracle(wl)
    d = _gpu(wl)
    o.step(steps)
    d.erf_rk3_step(steps)
    e = _errs(d.state(), o.state(), per_field=False)
    print(f"upwind-3 {case} {steps} steps:", e)
    assert all(v <= 1e-11 for v in e.values()), e


def test_mixed_upwind3_against_oracle():
    """FP32 perturbations with upwind-3 on a window of the scaling workload: the bounds of the
    other mixed-precision cases (1e-8 for rho, rho theta; 1e-6 for the momenta)."""
    wl = W.paper_scaling(nx=40, ny=36, nz=48)
    o = make_oracle(wl)
    d = _gpu(wl.with_(precision=W.PREC_MIXED32))
    o.step(20)
    d.erf_rk3_step(20)
    e = _errs(d.state(), o.state(), per_field=False)
    print("mixed upwind-3 paper_scaling 20 steps:", e)
    assert e["rho"] < 1e-8 and e["rhotheta"] < 1e-8, e
    assert max(e["rhou"], e["rhov"], e["rhow"]) < 1e-6, e


def test_tma_tiles_match_plain_loads_with_upwind3():
    from paper_2412_04395_gb300.erf import Dycore, ERF_OPT_TMA_STENCILS
    wl = W.paper_scaling(nx=128, ny=48, nz=32).with_(precision=W.PREC_MIXED32)
    a = _gpu(wl)
    b = _gpu(wl)
    b.erf_set_option(ERF_OPT_TMA_STENCILS, 0)
    assert a.erf_get_option(ERF_OPT_TMA_STENCILS) == 1
    a.erf_rk3_step(4)
    b.erf_rk3_step(4)
    sa, sb = a.state(), b.state()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f
