"""Pins of the anelastic oracle (Sec. 2.2 equations, Sec. 3.2 SSP-RK2 + projection; oracle/anelastic.py).

Fixed by something other than the oracle's own formulas:
  * the discrete Poisson operator div(grad) of the C-grid has the exact eigenmodes
    cos(2 pi k (i + 1/2) / nx) cos(2 pi l (j + 1/2) / ny) cos(pi m (k + 1/2) / nz) with eigenvalues
    -(4/dx^2) sin^2(pi k/nx) - (4/dy^2) sin^2(pi l/ny) - (4/dz^2) sin^2(pi m / (2 nz)) on a uniform
    grid with no-flux walls: the solver must return each mode from its image;
  * after a projection the discrete divergence of rho0 u vanishes, and projecting again changes
    nothing;
  * the anelastic constraint makes rho0 theta a conserved flux-form quantity and leaves a
    resting, unperturbed atmosphere at rest;
  * SSP-RK2 is second order in time (Shu & Osher 1988);
  * at low Mach number the anelastic and the compressible equations describe the same buoyant
    motion (Sec. 2.2): a 0.5 K bubble rises at the same speed in both within a few per cent.
"""
import numpy as np
import pytest

from oracle import anelastic as A
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle


def test_poisson_solver_inverts_the_discrete_eigenmodes():
    nx, ny, nz, dx, dy, dz = 16, 12, 10, 100.0, 150.0, 80.0
    i = np.arange(nx) + 0.5
    j = np.arange(ny) + 0.5
    k = np.arange(nz) + 0.5
    dzv = np.full(nz, dz)
    dzc = np.zeros(nz + 1)
    dzc[1:-1] = dz
    for kx, ky, m in ((1, 0, 0), (3, 2, 1), (0, 1, 4), (7, 5, 9), (0, 0, 2)):
        psi = (np.cos(np.pi * m * k / nz)[:, None, None] * np.cos(2 * np.pi * ky * j / ny)[None, :, None]
               * np.cos(2 * np.pi * kx * i / nx)[None, None, :])
        lam = (-4 / dx ** 2 * np.sin(np.pi * kx / nx) ** 2 - 4 / dy ** 2 * np.sin(np.pi * ky / ny) ** 2
               - 4 / dz ** 2 * np.sin(np.pi * m / (2 * nz)) ** 2)
        gx, gy, gz = A.gradient(psi, dx, dy, dzc)
        np.testing.assert_allclose(A.divergence(gx, gy, gz, dx, dy, dzv), lam * psi, atol=1e-15 * abs(lam))
        got = A.solve_poisson(lam * psi, dx, dy, dzv, dzc)
        if kx == ky == 0:
            got = got - got.mean() + psi.mean()      # the (0, 0) mode is defined up to a constant
        np.testing.assert_allclose(got, psi, atol=1e-12)


def bubble(nx=32, ny=4, nz=24, dx=200.0, amp=2.0, anelastic=1, **kw):
    zeta = W.uniform_zeta(nz, dx)
    X, Y, Z = W.cell_coords(nx, ny, zeta, dx, dx)
    r = np.sqrt(((X - 0.5 * nx * dx) / 1500.0) ** 2 + ((Z - 1500.0) / 1000.0) ** 2)
    dth = np.where(r < 1.0, amp * np.cos(0.5 * np.pi * r) ** 2, 0.0)
    base = dict(dt=2.0, n_substeps=6, closure=W.CLOSURE_NONE, dtheta=dth)
    base.update(kw)
    return W.Workload("bubble", nx, ny, nz, dx, dx, zeta, **base)


def an_oracle(wl):
    o = make_oracle(wl, anelastic=1)
    return o, A.Anelastic(o)


def test_projection_removes_the_divergence_and_is_idempotent():
    wl = bubble()
    o, a = an_oracle(wl)
    a.step(3)
    M = {k: o.get(k) for k in A.MOM}
    scale = np.abs(M["rhow"]).max() / wl.dx
    assert scale > 1e-4                                  # the bubble moves
    assert np.abs(a.div()).max() <= 1e-12 * scale
    M2, psi = a.project(M, wl.dt)
    for k in A.MOM:
        assert np.abs(M2[k] - M[k]).max() <= 1e-12 * np.abs(M["rhow"]).max()
    assert np.all(o.get("rho") == o.get("base_rho"))    # the density stays the base density


def test_rest_stays_at_rest_and_theta_is_conserved():
    wl = bubble(amp=0.0, brunt_N=0.01)
    o, a = an_oracle(wl)
    a.step(5)
    assert np.abs(o.get("rhow")).max() < 1e-12
    wl = bubble()
    o, a = an_oracle(wl)
    H = o.geom("Hc")
    m0 = float(np.sum(o.get("rhotheta") * H))
    a.step(6)
    assert abs(float(np.sum(o.get("rhotheta") * H)) - m0) <= 1e-13 * abs(m0)


def test_ssp_rk2_is_second_order_in_time():
    # a theta anomaly carried by a uniform wind without gravity: the flow stays divergence free
    # and the pressure zero; only the time integration differs between the runs
    def run(dt, T=40.0):
        wl = bubble(nx=24, nz=12, gravity=0.0, dt=dt, u=np.full((12, 4, 24), 15.0))
        o, a = an_oracle(wl)
        a.step(int(round(T / dt)))
        return o.get("rhotheta")
    ref = run(0.25)
    errs = [np.abs(run(dt) - ref).max() for dt in (4.0, 2.0, 1.0)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.8), (errs, orders)


def test_low_mach_bubble_rises_as_in_the_compressible_equations():
    amp, steps = 0.5, 30
    wl = bubble(nx=40, nz=30, amp=amp, dt=1.0)
    o, a = an_oracle(wl)
    a.step(steps)
    c = make_oracle(wl)
    c.step(steps)
    wa = o.get("rhow") / np.concatenate([o.get("rho")[:1], o.get("rho")])
    wc = c.get("rhow") / np.concatenate([c.get("rho")[:1], c.get("rho")])
    assert wa.max() > 0.05                                       # rising
    assert abs(wa.max() - wc.max()) < 0.05 * wc.max(), (wa.max(), wc.max())
    # the same pattern: the two vertical-velocity fields agree to ~10% in L2 (the compressible
    # run also carries the acoustic adjustment of its initial state, which is built at unchanged
    # pressure rather than at the base density)
    assert np.linalg.norm(wa - wc) < 0.12 * np.linalg.norm(wc)
