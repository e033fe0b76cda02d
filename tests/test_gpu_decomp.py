"""x-y pencil decomposition on the GPU path: every rank's window is a handle of its own on one
GPU, the halo strips move through erf_pack_columns / erf_unpack_columns between steps (the
single-process router; no kernel waits on another), and the assembled interiors must equal one
handle over the whole domain bit for bit, on the FP64 path (terrain, and an ABL with Smagorinsky,
MOST and Coriolis) and on the mixed-precision path."""
import numpy as np
import pytest
import torch

from paper_2412_04395_gb300 import decomp as D
from paper_2412_04395_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__ as ge
    ge.build()


def run_split(wl, px, py, steps):
    from paper_2412_04395_gb300.erf import Dycore
    whole = Dycore(wl)
    whole.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    whole.erf_rk3_step(steps)
    ref = whole.state()
    whole.close()
    dec = D.PencilDecomp(wl.nx, wl.ny, px, py, D.step_reach(wl.n_substeps, wl.terrain is not None))
    ranks = []
    for r in range(dec.size):
        w = D.window_workload(wl, dec, r)
        d = Dycore(w)
        d.erf_set_initial(w.dtheta, w.u, w.v, w.w)
        ranks.append(d)
    router = D.LocalRouter(dec, ranks)
    for _ in range(steps):
        for d in ranks:
            d.erf_rk3_step(1)
        router.exchange()
    torch.cuda.synchronize()
    got = D.gather_interior(dec, lambda r: ranks[r].state(), {f: ref[f].shape for f in FIELDS})
    windows = [ranks[r].state() for r in range(dec.size)]
    for d in ranks:
        d.close()
    return dec, ref, got, windows


@pytest.mark.parametrize("case", ["hill_fp64", "abl_fp64", "abl_mixed"])
def test_split_run_is_bit_identical_to_the_whole_domain(case):
    if case == "hill_fp64":
        wl, px, py = W.hill_bubble(nx=96, ny=80, nz=24, dx=50.0), 2, 1
    else:
        prec = W.PREC_FP64 if case == "abl_fp64" else W.PREC_MIXED32
        wl = W.abl_window(W.convective_abl, 2048, 2048, 300, 500, 64, 64, nz=40, precision=prec)
        px, py = 2, 2
    dec, ref, got, windows = run_split(wl, px, py, 4)
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), (case, f, float(np.abs(got[f] - ref[f]).max()))
    # after the last exchange every window (halo included) is the whole-domain state restricted
    for r in range(dec.size):
        for f in FIELDS:
            assert np.array_equal(windows[r][f], dec.window_slices(r, ref[f])), (case, r, f)


def test_column_block_round_trip_and_bounds():
    from paper_2412_04395_gb300.erf import Dycore, ErfError
    wl = W.density_current(nx=40, ny=6, nz=12, dx=400.0)
    d = Dycore(wl)
    d.erf_set_initial(wl.dtheta)
    d.erf_rk3_step(1)
    before = d.state()
    nb = d.erf_column_block_bytes(7, 3)
    assert nb == 8 * (4 * 12 + 13) * 7 * 3
    buf = d.pack(5, 7, 2, 3)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.array_equal(b[:12 * 21].reshape(12, 3, 7), before["rho"][:, 2:5, 5:12])
    assert np.array_equal(b[4 * 12 * 21:].reshape(13, 3, 7), before["rhow"][:, 2:5, 5:12])
    d.unpack(5, 7, 2, 3, torch.zeros_like(buf))
    after = d.state()
    assert np.all(after["rhotheta"][:, 2:5, 5:12] == 0.0)
    mask = np.ones(after["rho"].shape, bool)
    mask[:, 2:5, 5:12] = False
    assert np.array_equal(after["rho"][mask], before["rho"][mask])
    with pytest.raises(ErfError):
        d.pack(35, 7, 0, 1)            # beyond nx
    with pytest.raises(ErfError):
        d.pack(0, 1, -1, 2)
    d.close()
