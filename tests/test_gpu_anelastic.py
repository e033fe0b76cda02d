"""GPU parity of the anelastic equation set (Sec. 2.2) and its SSP-RK2 + projection time
integration (Sec. 3.2) against the oracle (oracle/anelastic.py), through the C ABI.

Bar: relative L2 <= 1e-11 for rho theta and the projection pressure p'; the momenta against the
momentum-vector norm (as the short compressible runs); the discrete divergence of the GPU's
momentum after the projection <= 1e-11 of the momentum scale; rest stays at rest.  Cases: a 2D-slab
warm bubble (inviscid) and a 3D bubble with Smagorinsky and Coriolis, on grids whose horizontal
sizes take the FFT's several radix-2 stages.
"""
import numpy as np
import pytest

from oracle import anelastic as A
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def bubble(nx, ny, nz, dx=200.0, amp=2.0, **kw):
    zeta = W.uniform_zeta(nz, dx)
    X, Y, Z = W.cell_coords(nx, ny, zeta, dx, dx)
    r = np.sqrt(((X - 0.5 * nx * dx) / 1500.0) ** 2 + (((Y - 0.5 * ny * dx) / 1500.0) ** 2 if ny > 4 else 0.0)
                + ((Z - 1500.0) / 1000.0) ** 2)
    dth = np.where(r < 1.0, amp * np.cos(0.5 * np.pi * r) ** 2, 0.0)
    base = dict(dt=2.0, n_substeps=6, closure=W.CLOSURE_NONE, dtheta=dth, anelastic=1)
    base.update(kw)
    return W.Workload("anelastic_bubble", nx, ny, nz, dx, dx, zeta, **base)


def run_both(wl, steps):
    from paper_2412_04395_gb300.erf import Dycore
    o = make_oracle(wl)
    a = A.Anelastic(o)
    a.step(steps)
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    d.erf_rk3_step(steps)
    return o, a, d


def compare(o, d):
    mom = np.sqrt(sum(np.linalg.norm(o.get(f)) ** 2 for f in A.MOM))
    gap = {"rhotheta": np.linalg.norm(d.erf_get_state("rhotheta") - o.get("rhotheta")) / np.linalg.norm(o.get("rhotheta")),
           "p_anelastic": np.linalg.norm(d.erf_get_state("p_anelastic") - o.get("p_anelastic"))
           / np.linalg.norm(o.get("p_anelastic"))}
    for f in A.MOM:
        gap[f] = np.linalg.norm(d.erf_get_state(f) - o.get(f)) / mom
    # rho stays each side's own base density (the two base states agree to round-off)
    rg = d.erf_get_state("rho")
    b = d.erf_get_state("base_rho")
    assert np.array_equal(rg, np.broadcast_to(b.reshape(-1, 1, 1) if b.ndim == 1 else b, rg.shape))
    assert np.array_equal(o.get("rho"), o.get("base_rho"))
    gap["rho"] = np.linalg.norm(rg - o.get("rho")) / np.linalg.norm(o.get("rho"))
    return gap


@pytest.mark.parametrize("case", ["slab", "3d_smagorinsky"])
def test_anelastic_parity(case):
    if case == "slab":
        wl, steps = bubble(64, 4, 32), 10
    else:
        wl, steps = bubble(32, 32, 24, closure=W.CLOSURE_SMAGORINSKY, f_cor=1e-4, u_g=5.0, v_g=0.0,
                           u=np.full((24, 32, 32), 5.0)), 6
    o, a, d = run_both(wl, steps)
    gap = compare(o, d)
    print(case, {k: "%.1e" % v for k, v in gap.items()})
    bad = {k: v for k, v in gap.items() if not v <= TOL}
    assert not bad, (bad, gap)
    # the GPU's momentum is divergence free after its projection
    M = {f: d.erf_get_state(f) for f in A.MOM}
    div = A.divergence(M["rhou"], M["rhov"], M["rhow"], a.dx, a.dy, a.dz)
    assert np.abs(div).max() <= 1e-11 * np.abs(M["rhow"]).max() / wl.dx
    assert np.abs(M["rhow"]).max() > 1e-3                                # the bubble rises
    d.close()


def test_anelastic_rest_stays_at_rest():
    from paper_2412_04395_gb300.erf import Dycore
    wl = bubble(32, 16, 20, amp=0.0, brunt_N=0.01)
    d = Dycore(wl)
    d.erf_set_initial()
    d.erf_rk3_step(10)
    assert np.abs(d.erf_get_state("rhow")).max() < 1e-12
    assert np.abs(d.erf_get_state("p_anelastic")).max() < 1e-9
    d.close()
