"""The windows behind the full-size parity tests (tests/test_gpu_full_size_windows.py), on the CPU.

* workloads.abl_window reproduces the full case's initial state on the chosen columns exactly,
  across the periodic seams;
* one RK3 step of the oracle reaches a bounded number of columns sideways: a 128-column window and
  a 176-column window around the same point give bit-identical fields on the central 80 x 80
  columns (24 columns in from the smaller window's edges), wider than the 32 x 32 centre the GPU
  comparison uses (48 columns in), for both ABL cases at their full-size levels and time steps.
"""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle


@pytest.mark.parametrize("case", [W.neutral_abl, W.convective_abl])
def test_window_is_the_full_case_restricted(case):
    full = case(nx=40, ny=36, nz=16)
    for i0, j0 in ((30, 28), (-5, -7), (3, 4)):
        w = W.abl_window(case, 40, 36, i0, j0, 16, 12, nz=16)
        ii = (i0 + np.arange(16)) % 40
        jj = (j0 + np.arange(12)) % 36
        assert np.array_equal(w.dtheta, full.dtheta[:, jj][:, :, ii])
        assert np.array_equal(w.u, full.u[:, jj][:, :, ii])
        assert np.array_equal(w.zeta, full.zeta) and w.dt == full.dt
        assert np.array_equal(w.knots[1], full.knots[1])


def test_smooth_velocity_window_is_the_field_restricted():
    u, v, w = W.smooth_velocity(40, 36, 12, 5, 1.0)
    a, b, c = W.smooth_velocity(40, 36, 12, 5, 1.0, i0=-7, j0=30, nx=16, ny=10)
    ii = (-7 + np.arange(16)) % 40
    jj = (30 + np.arange(10)) % 36
    for full, win in ((u, a), (v, b), (w, c)):
        np.testing.assert_allclose(win, full[:, jj][:, :, ii], rtol=0, atol=1e-15)
    assert w.shape == (13, 36, 40) and np.all(w[0] == 0) and np.all(w[-1] == 0)
    assert 0.2 < np.std(u) < 2.0


@pytest.mark.parametrize("case,n_full", [(W.neutral_abl, 1024), (W.convective_abl, 2048)])
def test_one_step_reach_is_inside_the_window_margin(case, n_full):
    def step(n):
        wl = W.abl_window(case, n_full, n_full, -(n // 2), -(n // 2), n, n)
        o = make_oracle(wl)
        o.step(1)
        return o.state()

    a, b = step(128), step(176)
    h = 40
    for f in a:
        assert np.array_equal(a[f][:, 64 - h:64 + h, 64 - h:64 + h], b[f][:, 88 - h:88 + h, 88 - h:88 + h]), f
