"""Pins of the oracle's Deardorff 1.5-order closure (closure 4; Sec. 2.3, coefficients of Moeng
1984 as App. D states) and of its Rayleigh damping (Sec. 3.7; App. D: an inverse timescale ramped
by sin^2 from 0 at the bottom of the damping layer to its value at the top).

Each pin is fixed by something other than the oracle's own formulas:
  * uniform SGS energy e in neutral air: l = Delta, so Deardorff's viscosity is the constant
    0.1 Delta sqrt(e) and its heat diffusivity (1 + 2) times that - the tendencies must equal the
    constant-nu closure with nu = 0.1 Delta sqrt(e) and Pr_t = 1/3;
  * pure dissipation at rest: de/dt = -C_eps e^(3/2) / Delta with C_eps = 0.19 + 0.51 = 0.70 has the
    exact solution e(t) = (e0^(-1/2) + C_eps t / (2 Delta))^(-2); the RK3 steps converge to it at
    second order (the low-storage RK3 of Sec. 3.1 is third order for linear problems only, and
    this decay is nonlinear);
  * linear shear u = S z: S_13 = S/2 is the only strain, so the production is 2 K_m (2 (S/2)^2) =
    K_m S^2;
  * stable linear stratification with small e: the length scale switches to 0.76 sqrt(e)/N, the
    buoyancy term is -K_h N^2;
  * the diffusion of e is a flux divergence with no wall flux: it sums to zero over the domain;
  * Rayleigh damping of a uniform wind offset at rest: each RK3 step multiplies the offset by the
    RK3 amplification factor of du/dt = -tau u, 1 - h + h^2/2 - h^3/6 (h = tau dt); the rate is 0
    below the layer, tau_max at the top, tau_max/2 at mid-layer, and grows monotonically;
  * a state at the reference (u = u_g, theta = theta0) is not damped.
"""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle


def rest_case(nx=8, ny=8, nz=24, dz=10.0, **kw):
    zeta = W.uniform_zeta(nz, dz)
    base = dict(dt=0.5, n_substeps=6, closure=W.CLOSURE_DEARDORFF, Pr_t=1.0 / 3.0)
    base.update(kw)
    return W.Workload("rest", nx, ny, nz, dz, dz, zeta, **base)


def test_uniform_tke_neutral_equals_constant_viscosity():
    nz, dz = 16, 10.0
    X, Y, Z = W.cell_coords(16, 12, W.uniform_zeta(nz, dz), dz, dz)
    u = 2.0 * np.sin(2 * np.pi * X / 160.0) * np.cos(2 * np.pi * Z / 320.0)
    v = 1.0 * np.cos(2 * np.pi * Y / 120.0)
    dth = 0.3 * np.sin(2 * np.pi * X / 160.0) * np.sin(2 * np.pi * Y / 120.0) * np.exp(-Z / 80.0)
    e0 = 0.4
    wl = rest_case(16, 12, nz, dz, gravity=0.0, u=u, v=v, dtheta=dth, tke=np.full((nz, 12, 16), e0))
    o4 = make_oracle(wl)
    r4 = o4.slow_rhs()
    Km = 0.1 * dz * np.sqrt(e0)                  # Delta = (dx dy dz)^(1/3) = dz
    o1 = make_oracle(wl.with_(closure=W.CLOSURE_CONST_NU, nu=Km, Pr_t=1.0 / 3.0))
    r1 = o1.slow_rhs()
    for k in ("R_rhou", "R_rhov", "R_rhow", "R_rhotheta"):
        scale = np.abs(r1[k]).max()
        assert np.abs(r4[k] - r1[k]).max() <= 1e-12 * scale, k
    np.testing.assert_allclose(o4.aux("mu"), o4.get("rho") * Km, rtol=1e-14)
    np.testing.assert_allclose(o4.aux("muh"), 3.0 * o4.get("rho") * Km, rtol=1e-14)


def _decay(e0, dt, t_end, Delta=10.0):
    wl = rest_case(dt=dt, tke=np.full((24, 8, 8), e0))
    o = make_oracle(wl)
    for _ in range(int(round(t_end / dt))):
        o.step(1)
    return o.get("rhotke") / o.get("rho")


def test_dissipation_follows_the_exact_decay_at_second_order():
    e0, T, Delta = 2.0, 40.0, 10.0
    exact = (e0 ** -0.5 + 0.70 * T / (2.0 * Delta)) ** -2
    errs = []
    for dt in (1.0, 0.5, 0.25):
        e = _decay(e0, dt, T)
        assert np.ptp(e) <= 1e-13 * exact       # stays uniform at rest
        errs.append(float(e.mean()) - exact)
    errs = np.array(errs)
    assert np.all(errs > 0) and abs(errs[-1]) < 1e-5 * exact
    orders = np.log2(errs[:-1] / errs[1:])
    assert orders[-1] > 1.8 and np.all(orders > 1.5), orders


def test_linear_shear_production():
    nz, dz, S, e0 = 20, 10.0, 0.02, 0.3
    zc = 0.5 * (W.uniform_zeta(nz, dz)[:-1] + W.uniform_zeta(nz, dz)[1:])
    u = np.broadcast_to((S * zc)[:, None, None], (nz, 8, 8)).copy()
    wl = rest_case(nz=nz, dz=dz, gravity=0.0, u=u, tke=np.full((nz, 8, 8), e0))
    o = make_oracle(wl)
    o.slow_rhs()
    rho = o.get("rho")
    Km = 0.1 * dz * np.sqrt(e0)
    eps = 0.70 * e0 ** 1.5 / dz
    want = rho * (Km * S * S - eps)
    src = o.aux("tke_src")
    # interior levels: the cells next to the slip walls see half the edge strain
    np.testing.assert_allclose(src[2:-2], want[2:-2], rtol=1e-12)


def test_stable_stratification_switches_the_length_scale():
    nz, dz, gam, e0 = 24, 10.0, 0.01, 0.01      # theta = 300 + 0.01 z: N ~ 0.018 1/s
    top = nz * dz
    knots = (np.array([0.0, top]), np.array([300.0, 300.0 + gam * top]))
    wl = rest_case(nz=nz, dz=dz, knots=knots, tke=np.full((nz, 8, 8), e0))
    o = make_oracle(wl)
    o.slow_rhs()
    rho, th = o.get("rho"), o.get("rhotheta") / o.get("rho")
    N2 = 9.81 / th * gam
    l = 0.76 * np.sqrt(e0) / np.sqrt(N2)
    assert np.all(l < dz)                       # the stable length scale is the shorter
    Km = 0.1 * l * np.sqrt(e0)
    Kh = (1.0 + 2.0 * l / dz) * Km
    eps = (0.19 + 0.51 * l / dz) * e0 ** 1.5 / l
    want = rho * (-Kh * N2 - eps)
    np.testing.assert_allclose(o.aux("tke_src")[1:-1], want[1:-1], rtol=1e-10)
    np.testing.assert_allclose(o.aux("muh")[1:-1], (rho * Kh)[1:-1], rtol=1e-10)


def test_tke_diffusion_conserves():
    nz, dz = 16, 10.0
    X, Y, Z = W.cell_coords(12, 10, W.uniform_zeta(nz, dz), dz, dz)
    e = 0.2 + 0.15 * np.sin(2 * np.pi * X / 120.0) * np.cos(np.pi * Z / 160.0) + 0.05 * np.cos(2 * np.pi * Y / 100.0)
    wl = rest_case(12, 10, nz, dz, tke=e)
    o = make_oracle(wl)
    o.slow_rhs()
    rho = o.get("rho")
    # the local part of the source at rest in neutral air: -rho eps with l = Delta
    local = -rho * 0.70 * e ** 1.5 / dz
    diff = o.aux("tke_src") - local
    assert abs(diff.sum()) <= 1e-12 * np.abs(diff).sum()
    assert np.abs(diff).max() > 1e-6                          # it is not trivially zero


def test_tke_stays_non_negative():
    e = _decay(0.5, 30.0, 90.0, Delta=10.0)    # dissipation far faster than the step resolves
    assert np.all(e >= 0.0)


# ------------------------------------------------------------------ Rayleigh damping
def ray_case(nz=40, dz=25.0, **kw):
    zeta = W.uniform_zeta(nz, dz)
    base = dict(dt=1.0, n_substeps=6, closure=W.CLOSURE_NONE, gravity=9.81, u_g=10.0, brunt_N=0.01,
                ray_tau=0.05, ray_zd=600.0, ray_fields=W.RAY_U | W.RAY_V | W.RAY_W | W.RAY_THETA)
    base.update(kw)
    return W.Workload("ray", 6, 6, nz, 100.0, 100.0, zeta, **base)


def u_damping_rates(nz=40, dz=25.0, delta=1.5):
    """Per-level damping rate of a uniform wind offset, from the offset's decay over one RK3 step
    (the inverse of the RK3 amplification factor 1 - h + h^2/2 - h^3/6, h = rate dt)."""
    wl = ray_case(nz, dz, u=np.full((nz, 6, 6), 10.0 + delta))
    o = make_oracle(wl)
    u0 = o.get("rhou") / o.get("rho")
    o.step(1)
    rho = o.get("rho")
    off = o.get("rhou") / rho - 10.0
    rate = np.empty(nz)
    for k in range(nz):
        a = off[k].mean() / (u0[k].mean() - 10.0)     # amplification factor at level k
        assert np.ptp(off[k]) <= 1e-12
        # invert 1 - h + h^2/2 - h^3/6 = a for h = tau dt (monotone on [0, 1])
        lo, hi = 0.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if 1 - mid + mid * mid / 2 - mid ** 3 / 6 > a:
                lo = mid
            else:
                hi = mid
        rate[k] = 0.5 * (lo + hi) / wl.dt
    return wl, rate


def test_rayleigh_decay_of_a_uniform_wind_offset_is_the_rk3_factor():
    nz, dz = 40, 25.0
    wl, rate = u_damping_rates(nz, dz)
    zc = (np.arange(nz) + 0.5) * dz
    top = nz * dz
    assert np.all(rate[zc <= wl.ray_zd] < 1e-12)
    assert np.all(np.diff(rate[zc > wl.ray_zd]) > 0)
    # tau_max at the top and tau_max / 2 at mid-layer: the ramp through the cell centres, whose
    # heights straddle those points, brackets both values
    zm = 0.5 * (wl.ray_zd + top)
    k_mid = np.searchsorted(zc, zm)
    assert rate[k_mid - 1] < 0.5 * wl.ray_tau < rate[k_mid]
    assert 0.95 * wl.ray_tau < rate[-1] <= wl.ray_tau
    # the ramp starts flat (sin^2): the rate one cell into the layer is second order in its depth
    k0 = np.searchsorted(zc, wl.ray_zd)
    frac = (zc[k0] - wl.ray_zd) / (top - wl.ray_zd)
    assert rate[k0] < 3.0 * wl.ray_tau * frac ** 2


def test_rayleigh_leaves_the_reference_state_alone():
    nz = 40
    wl = ray_case(nz, u=np.full((nz, 6, 6), 10.0))
    on = make_oracle(wl).slow_rhs()
    off = make_oracle(wl.with_(ray_fields=0)).slow_rhs()
    for k in on:
        assert np.array_equal(on[k], off[k]), k


def test_rayleigh_theta_relaxes_toward_the_base_state():
    nz = 40
    X, Y, Z = W.cell_coords(6, 6, W.uniform_zeta(nz, 25.0), 100.0, 100.0)
    dth = 0.5 * np.cos(2 * np.pi * X / 600.0)
    wl = ray_case(nz, dtheta=dth, u=np.full((nz, 6, 6), 10.0))
    o = make_oracle(wl)
    on = o.slow_rhs()
    off = make_oracle(wl.with_(ray_fields=0)).slow_rhs()
    d = on["R_rhotheta"] - off["R_rhotheta"]
    rho = o.get("rho")
    th = o.get("rhotheta") / rho
    th0 = o.get("base_theta")
    excess = rho * (th - th0)
    zc = (np.arange(nz) + 0.5) * 25.0
    up = zc > wl.ray_zd
    assert np.all(d[~up] == 0.0)
    live = np.abs(dth[0]) > 1e-3                   # columns with a theta excess
    ratio = -d[up][:, live] / excess[up][:, live]  # the local rate, positive: toward theta0
    assert np.all(ratio > 0)
    # the same rate at every column of a level, and zero change where there is no excess
    assert np.all(np.ptp(ratio, axis=1) <= 1e-9 * ratio.max(axis=1))
    assert np.all(np.abs(d[up][:, ~live]) <= 1e-12 * np.abs(d).max())
    # theta is damped at the rate the wind offset decays at, level by level (one ramp for all)
    _, rate_u = u_damping_rates(nz, 25.0)
    np.testing.assert_allclose(ratio.mean(axis=1), rate_u[up], rtol=1e-9)
