"""GPU parity of the Deardorff 1.5-order closure and of Rayleigh damping (FP64 path) against the
oracle, through the C ABI, element by element.

Bar: relative L2 <= 1e-11 per field (rho e included), or, for the short runs, 3 x the oracle's own
round-off floor where that is larger (the normalisation of tests/test_gpu_parity.py).  Cases:
  * a convective-ABL window (MOST, Coriolis) with the Deardorff closure and an SGS energy profile
    decreasing with height, 10 steps;
  * the same with Rayleigh damping of u, v, w and theta in the upper third;
  * the warm bubble over the Gaussian hill with Rayleigh damping of every field (terrain), 20 steps;
  * the oracle's closed forms on the GPU: pure dissipation at rest matches the oracle to round-off;
  * the decomposition's column blocks carry rho e (split run bit-identical to the whole domain).
"""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle
from test_gpu_parity import _errors, _ulp_floor, TOL, FIELDS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def _tke_profile(wl):
    zc = 0.5 * (wl.zeta[:-1] + wl.zeta[1:])
    e = 0.6 * np.exp(-zc / 300.0) + 0.01
    return np.broadcast_to(e[:, None, None], (wl.nz, wl.ny, wl.nx)).copy()


def _gpu(wl):
    from paper_2412_04395_gb300.erf import Dycore
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if wl.closure == W.CLOSURE_DEARDORFF and wl.tke is not None:
        d.erf_set_state("rhotke", d.erf_get_state("rho") * wl.tke)
    return d


def _parity(wl, steps, tke=False):
    o = make_oracle(wl)
    d = _gpu(wl)
    o.step(steps)
    d.erf_rk3_step(steps)
    ref = o.state()
    gap = _errors(d.state(), ref)
    floor = _ulp_floor(wl, steps, ref)
    bad = {f: (gap[f], floor[f]) for f in FIELDS if not gap[f] <= max(TOL, 3.0 * floor[f])}
    assert not bad, (bad, gap, floor)
    if tke:
        a, b = d.erf_get_state("rhotke"), o.get("rhotke")
        e = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        assert e <= TOL, e
        assert np.all(a >= 0.0)
        gap["rhotke"] = e
    diag = d.erf_diagnostics()
    assert diag["status"] == 0, diag
    d.close()
    return gap


def _abl(**kw):
    wl = W.abl_window(W.convective_abl, 2048, 2048, 700, 900, 40, 36, nz=40, precision=W.PREC_FP64)
    wl = wl.with_(closure=W.CLOSURE_DEARDORFF, Pr_t=1.0 / 3.0, **kw)
    return wl.with_(tke=_tke_profile(wl))


def test_deardorff_convective_abl_window():
    gap = _parity(_abl(), 10, tke=True)
    print("Deardorff convective ABL, 10 steps:", gap)


def test_deardorff_with_rayleigh_damping():
    wl = _abl(ray_tau=0.02, ray_zd=1000.0, ray_fields=W.RAY_U | W.RAY_V | W.RAY_W | W.RAY_THETA)
    gap = _parity(wl, 10, tke=True)
    print("Deardorff + Rayleigh, 10 steps:", gap)


def test_rayleigh_over_terrain():
    wl = W.hill_bubble(nx=48, ny=40, nz=40, dx=100.0, dz0=40.0, ratio=1.03)
    wl = wl.with_(ray_tau=0.05, ray_zd=0.6 * wl.zeta[-1], ray_fields=W.RAY_U | W.RAY_V | W.RAY_W | W.RAY_THETA)
    gap = _parity(wl, 20)
    print("hill bubble + Rayleigh, 20 steps:", gap)
    # damping changes the run (it is not a no-op on the GPU)
    from paper_2412_04395_gb300.erf import Dycore
    a = _gpu(wl)
    b = _gpu(wl.with_(ray_fields=0))
    a.erf_rk3_step(20)
    b.erf_rk3_step(20)
    assert not np.array_equal(a.erf_get_state("rhow"), b.erf_get_state("rhow"))


def test_pure_dissipation_at_rest_matches_the_oracle():
    zeta = W.uniform_zeta(24, 10.0)
    wl = W.Workload("rest", 16, 8, 24, 10.0, 10.0, zeta, dt=1.0, n_substeps=6,
                    closure=W.CLOSURE_DEARDORFF, tke=np.full((24, 8, 16), 2.0))
    o = make_oracle(wl)
    d = _gpu(wl)
    o.step(10)
    d.erf_rk3_step(10)
    e_gpu = d.erf_get_state("rhotke") / d.erf_get_state("rho")
    e_orc = o.get("rhotke") / o.get("rho")
    assert np.abs(e_gpu - e_orc).max() <= 1e-13 * e_orc.max()
    exact = (2.0 ** -0.5 + 0.70 * 10.0 / (2.0 * 10.0)) ** -2
    assert abs(e_gpu.mean() - exact) < 1e-3 * exact


def test_split_run_carries_the_sgs_energy():
    import torch
    from paper_2412_04395_gb300 import decomp as D
    from paper_2412_04395_gb300.erf import Dycore
    wl = W.abl_window(W.convective_abl, 2048, 2048, 100, 100, 64, 32, nz=24, precision=W.PREC_FP64)
    wl = wl.with_(closure=W.CLOSURE_DEARDORFF, Pr_t=1.0 / 3.0)
    wl = wl.with_(tke=_tke_profile(wl))
    steps = 3
    whole = _gpu(wl)
    whole.erf_rk3_step(steps)
    ref = whole.erf_get_state("rhotke")
    dec = D.PencilDecomp(wl.nx, wl.ny, 2, 1, D.step_reach(wl.n_substeps, False))
    ranks = []
    for r in range(2):
        kw = {n: dec.window_slices(r, getattr(wl, n)) for n in ("dtheta", "u", "tke")}
        ranks.append(_gpu(wl.with_(nx=dec.pencil(r).nxw, **kw)))
    router = D.LocalRouter(dec, ranks)
    for _ in range(steps):
        for d in ranks:
            d.erf_rk3_step(1)
        router.exchange()
    torch.cuda.synchronize()
    got = D.gather_interior(dec, lambda r: {"rhotke": ranks[r].erf_get_state("rhotke")}, {"rhotke": ref.shape})
    assert np.array_equal(got["rhotke"], ref)
