"""Pins of the passive scalar of the oracle (Sec. 3.1: scalars are advanced after the acoustic
substeps with the stage-averaged normal momenta that advanced rho).

* consistency with continuity: phi = 1 stays 1 to round-off, with substeps (where the averaged
  fluxes differ from the stage ones), over terrain and with no substeps;
* conservation of the tracer mass (flux form, periodic sides, walls);
* a resting atmosphere leaves any tracer unchanged bit for bit;
* uniform translation converges to the exactly translated cell averages (observed order)."""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle


def _ratio_err(o):
    return float(np.max(np.abs(o.get("rhophi") / o.get("rho") - 1.0)))


@pytest.mark.parametrize("case", ["density_current", "hill", "abl", "nosub"])
def test_phi_one_stays_one(case):
    if case == "density_current":
        wl = W.density_current(nx=64, ny=4, nz=32, dx=200.0)
        n = 8
    elif case == "hill":
        wl = W.hill_bubble(nx=24, ny=24, nz=32, dx=100.0)
        n = 4
    elif case == "abl":
        wl = W.neutral_abl(nx=16, ny=16, nz=24, dx=20.0).with_(precision=W.PREC_FP64)
        n = 4
    else:
        wl = W.density_current(nx=64, ny=4, nz=32, dx=200.0)
        n = 4
    wl = W.with_tracer(wl, "one")
    over = {"substep_mode": 1} if case == "nosub" else {}
    if case == "nosub":
        wl = wl.with_(dt=0.05)
    o = make_oracle(wl, **over)
    o.step(n)
    assert _ratio_err(o) < 2e-13


def test_tracer_mass_is_conserved():
    wl = W.with_tracer(W.hill_bubble(nx=24, ny=24, nz=32, dx=100.0), "blob", radius_frac=0.25)
    o = make_oracle(wl)
    vol = o.geom("Hc")
    m0 = float(np.sum(o.get("rhophi") * vol))
    o.step(5)
    m1 = float(np.sum(o.get("rhophi") * vol))
    assert abs(m1 - m0) / m0 < 1e-13


def test_tracer_at_rest_is_unchanged():
    wl = W.hill_bubble(nx=16, ny=16, nz=24, dx=100.0).with_(dtheta=None)
    wl = W.with_tracer(wl, "blob", radius_frac=0.3)
    o = make_oracle(wl)
    q0 = o.get("rhophi")
    o.step(3)
    assert np.array_equal(o.get("rhophi"), q0)


def _translate_error(nx, scheme):
    L, U = 6400.0, 10.0
    dx = L / nx
    zeta = np.arange(3) * 100.0
    wl = W.Workload("box", nx, 1, 2, dx, dx, zeta, gravity=0.0, dt=dx / 200.0, scal_adv=scheme)
    xf = np.arange(nx) * dx
    u = np.full((2, 1, nx), U)
    k = 2 * np.pi / L
    # phi given as cell averages of 1 + 0.5 sin(kx)
    avg = lambda x0: 1.0 + 0.5 * (np.cos(k * x0) - np.cos(k * (x0 + dx))) / (k * dx)
    phi = np.broadcast_to(avg(xf)[None, None, :], (2, 1, nx)).copy()
    wl = wl.with_(u=u, tracer=1, phi=phi)
    o = make_oracle(wl)
    T = L / U / 4
    steps = int(round(T / wl.dt))
    o.step(steps)
    ex = avg(xf - U * steps * wl.dt)
    got = (o.get("rhophi") / o.get("rho"))[0, 0]
    return float(np.max(np.abs(got - ex)))


@pytest.mark.parametrize("scheme", [0, 1])
def test_tracer_translation_converges(scheme):
    ns = [32, 64, 128]
    errs = [_translate_error(n, scheme) for n in ns]
    order = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert order > 2.5, (errs, order)
