"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Every test here checks the oracle against something other than itself: coefficients expanded
by hand from the printed formulas (tests/golden), closed forms, exact discrete eigenvalues,
invariants (mass, rest state), dispersion relations and measured orders of accuracy.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RD, CP = 287.0, 1004.5
CV = CP - RD
GAMMA = CP / CV


def _golden_interp():
    rows = []
    for line in open(os.path.join(GOLD, "interpolants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        rows.append((t[0], float(t[1]), float(t[2]), [float(x) for x in t[3:9]]))
    return rows


ORDER = {"centred2": 2, "centred4": 4, "centred6": 6, "upwind3": 3, "upwind5": 5}


@pytest.mark.parametrize("row", _golden_interp(), ids=lambda r: f"{r[0]}{r[1]:+.0f}")
def test_interpolant_weights_match_printed_formulas(row):
    """Sec. 3.6: the oracle's interpolants reproduce the hand-expanded weights exactly."""
    name, s, den, num = row
    for m in range(6):
        e = np.zeros(6); e[m] = 1.0
        assert oracle.interp(e, s, ORDER[name]) == pytest.approx(num[m] / den, abs=1e-15)
    assert sum(num) / den == pytest.approx(1.0, abs=1e-15)


def _cell_avgs_of_poly(coef, h=1.0, x0=0.0):
    """Cell averages over [m - 1/2, m + 1/2] (m = -3..2, scaled by h) of sum coef[n] x^n;
    the interface m - 1/2 for m = 0 sits at x = -h/2 + x0."""
    P = np.polynomial.Polynomial(coef).integ()
    q = []
    for m in range(-3, 3):
        a, b = x0 + (m - 0.5) * h, x0 + (m + 0.5) * h
        q.append((P(b) - P(a)) / h)
    exact = np.polynomial.Polynomial(coef)(x0 - 0.5 * h)
    return np.array(q), exact


@pytest.mark.parametrize("order,deg", [(2, 1), (3, 2), (4, 3), (5, 4), (6, 5)])
def test_interpolants_exact_for_polynomials(order, deg):
    """Reconstruction from cell averages is exact up to degree order-1 and not beyond."""
    rng = np.random.default_rng(7)
    for s in (1.0, -1.0):
        for trial in range(5):
            coef = rng.normal(size=deg + 1)
            q, ex = _cell_avgs_of_poly(coef)
            assert oracle.interp(q, s, order) == pytest.approx(ex, abs=1e-12)
        # one degree higher is not reproduced
        coef = np.zeros(deg + 2); coef[-1] = 1.0
        q, ex = _cell_avgs_of_poly(coef)
        assert abs(oracle.interp(q, s, order) - ex) > 1e-6


def test_weno5_linear_weights_on_linear_data_and_exact_on_quadratics():
    """Jiang-Shu 1996: equal smoothness indicators (linear data) give the linear weights, which
    recombine to the upwind-5 interpolant; every candidate is exact for quadratics."""
    rng = np.random.default_rng(3)
    for s in (1.0, -1.0):
        for z in (False, True):
            q = 300.0 + 0.7 * np.arange(6) - 2.0
            assert oracle.weno5(q, s, z) == pytest.approx(oracle.interp(q, s, 5), abs=1e-12)
            for trial in range(5):
                coef = rng.normal(size=3)
                qq, ex = _cell_avgs_of_poly(coef)
                assert oracle.weno5(qq, s, z) == pytest.approx(ex, abs=1e-12)


def test_weno5_no_new_extremum_at_a_step():
    """Across a discontinuity the reconstruction stays inside the data range (essentially
    non-oscillatory); the linear upwind-5 interpolant overshoots on the same data."""
    for s in (1.0, -1.0):
        for jump in range(1, 6):
            q = np.where(np.arange(6) < jump, 300.0, 310.0)
            v = oracle.weno5(q, s)
            assert 300.0 - 1e-3 <= v <= 310.0 + 1e-3
    q = np.array([300.0, 300.0, 300.0, 310.0, 310.0, 310.0])
    lin = oracle.interp(q, 1.0, 5)
    assert lin < 300.0 - 0.1 or lin > 310.0 + 0.1 or abs(oracle.weno5(q, 1.0) - 300.0) < abs(lin - 300.0)


def test_eos_closed_forms():
    """Sec. 2.1: p = P00 (R_d rho theta/P00)^gamma; pi = (p/P00)^(R_d/c_p) so p = R_d rho theta pi;
    sound speed sqrt(gamma p/rho) ~ 347 m/s at 300 K, 1000 hPa."""
    p, pi = oracle.eos(1.0e5 / RD)
    assert p == pytest.approx(1.0e5, rel=1e-15) and pi == pytest.approx(1.0, rel=1e-15)
    rt = 1.2 * 290.0
    p, pi = oracle.eos(rt)
    assert p == pytest.approx(RD * rt * pi, rel=1e-14)
    rho = 1.0e5 / (RD * 300.0)
    p, _ = oracle.eos(rho * 300.0)
    h = 1e-6 * rho * 300.0
    dpdrt = (oracle.eos(rho * 300.0 + h)[0] - oracle.eos(rho * 300.0 - h)[0]) / (2 * h)
    assert dpdrt == pytest.approx(GAMMA * p / (rho * 300.0), rel=1e-8)   # dp/d(rho theta) = gamma p/(rho theta)
    c = np.sqrt(GAMMA * p / rho)
    assert 346.0 < c < 348.5


def test_thomas_against_dense_solve():
    rng = np.random.default_rng(11)
    for n in (1, 2, 5, 63, 127):
        a = rng.uniform(-1, 1, n); c = rng.uniform(-1, 1, n)
        b = 2.5 + rng.uniform(0, 1, n)
        d = rng.normal(size=n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x = oracle.thomas(a, b, c, d)
        np.testing.assert_allclose(x, np.linalg.solve(A, d), rtol=1e-13, atol=1e-13)
        assert np.max(np.abs(A @ x - d)) < 1e-13


def test_hse_column_residual_and_adiabatic_closed_form():
    """Sec. 3.8 Newton-Raphson HSE: discrete residual ~ round-off; for constant theta the
    continuous solution is pi(z) = pi_s - g z/(c_p theta), approached at second order."""
    g = 9.81
    errs = []
    for dz in (200.0, 100.0, 50.0):
        zc = (np.arange(int(6000 / dz)) + 0.5) * dz
        th = np.full_like(zc, 300.0)
        rho, p = oracle.hse_column(zc, th, 1.0e5, 300.0, g)
        zprev = np.concatenate([[0.0], zc[:-1]])
        pprev = np.concatenate([[1.0e5], p[:-1]])
        rs = 1.0e5 ** (1 / GAMMA) * 1.0e5 ** (1 - 1 / GAMMA) / (RD * 300.0)
        rprev = np.concatenate([[rs], rho[:-1]])
        res = p - pprev + 0.5 * g * (zc - zprev) * (rprev + rho)
        assert np.max(np.abs(res) / p) < 1e-12
        pi_exact = 1.0 - g * zc / (CP * 300.0)
        p_exact = 1.0e5 * pi_exact ** (CP / RD)
        errs.append(np.max(np.abs(p - p_exact) / p_exact))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2
    # stable stratification: theta0 = 300 exp(N^2 z/g) gives rho decreasing and dp/dz = -rho g
    zc = (np.arange(40) + 0.5) * 100.0
    th = 300.0 * np.exp(1e-4 * zc / g)
    rho, p = oracle.hse_column(zc, th, 1.0e5, 300.0, g)
    assert np.all(np.diff(rho) < 0) and np.all(np.diff(p) < 0)


def test_base_state_matches_eos_and_rest_is_exact():
    """p0 = EOS(rho0 theta0) so the undisturbed state has p' = 0 bit for bit."""
    wl = W.hill_bubble(nx=16, ny=12, nz=10, dx=400.0, dz0=150.0, ratio=1.02, h0=300.0).with_(dtheta=None)
    o = make_oracle(wl)
    r = o.slow_rhs()
    assert np.all(r["pp"] == 0.0)
    for k in ("R_rho", "R_rhotheta", "R_rhou", "R_rhov", "R_rhow"):
        assert np.all(r[k] == 0.0), k


def test_terrain_metrics_reduce_on_flat_and_are_consistent():
    """App. B: flat terrain -> identity metrics; heights telescope; 4th-order h_xi at w-faces."""
    wl = W.hill_bubble(nx=32, ny=8, nz=6, dx=250.0, dz0=100.0, ratio=1.0, terrain=False)
    o = make_oracle(wl, init=False)
    dz = np.diff(wl.zeta)
    assert np.all(o.geom("Hc") == dz[:, None, None]) and np.all(o.geom("Hx") == dz[:, None, None])
    assert np.all(o.geom("hxi_w") == 0.0) and np.all(o.geom("hxi_x") == 0.0)
    # periodic sinusoidal terrain in x: h = A sin(2 pi x/L); metrics converge to the analytic slope
    errs = []
    for nx in (16, 32, 64):
        dx = 8000.0 / nx
        x = np.arange(nx) * dx
        h = 100.0 * np.sin(2 * np.pi * x / 8000.0)
        ter = np.tile(h, (4, 1))
        zeta = np.linspace(0.0, 2000.0, 5)
        wl2 = W.Workload("t", nx, 4, 4, dx, dx, zeta, terrain=ter, terrain_beta=1)
        o = make_oracle(wl2, init=False)
        Hc = o.geom("Hc")
        # column heights telescope to z_t - <h> (4-node average of h at the cell centre)
        hcell = 0.5 * (h + np.roll(h, -1))
        np.testing.assert_allclose(Hc.sum(axis=0)[0], 2000.0 - hcell, rtol=0, atol=1e-9)
        # h_xi at the w-face k=0 (terrain surface) vs analytic slope at the cell centre
        xc = x + 0.5 * dx
        exact = 100.0 * (2 * np.pi / 8000.0) * np.cos(2 * np.pi * xc / 8000.0)
        # the face height is a 4-node average: slope of the averaged sine
        exact *= np.cos(np.pi * dx / 8000.0)
        errs.append(np.max(np.abs(o.geom("hxi_w")[0, 0] - exact)))
    assert np.log2(errs[0] / errs[1]) > 3.7 and np.log2(errs[1] / errs[2]) > 3.7


def test_mass_conserved_to_roundoff():
    """Sec. 4.1.2: total mass conserved to machine precision on closed/periodic domains."""
    wl = W.density_current(nx=48, ny=4, nz=24, dx=250.0, steps=5)
    o = make_oracle(wl)
    m0 = o.mass()
    for n in range(5):
        o.step(1)
        m1 = o.mass()
        assert abs(m1 - m0) / m0 < 1e-14
    wl = W.hill_bubble(nx=16, ny=16, nz=16, dx=250.0, dz0=100.0, ratio=1.03, h0=300.0)
    o = make_oracle(wl, u=None)
    o.set_initial(wl.dtheta, np.full(o.shape_c, 4.0), np.full(o.shape_c, -2.0), None)
    m0 = o.mass()
    o.step(4)
    assert abs(o.mass() - m0) / m0 < 4e-14


def test_mass_sum_is_the_exactly_rounded_sum():
    """The domain mass is the sum of rho times the cell volumes; the oracle's compensated sum
    equals math.fsum (exactly rounded) of the same products to within an ulp, on a field whose
    plain running sum already loses more than that."""
    import math
    wl = W.hill_bubble(nx=64, ny=64, nz=48, dx=250.0, dz0=60.0, ratio=1.03, h0=300.0)
    o = make_oracle(wl)
    rng = np.random.default_rng(5)
    o.set("rho", o.get("rho") * (1.0 + 0.3 * rng.standard_normal(o.shape_c)))
    terms = (o.get("rho") * o.geom("Hc") * wl.dx * wl.dy).ravel()
    exact = math.fsum(terms)
    assert abs(o.mass() - exact) <= 2.3e-16 * exact
    plain = 0.0
    for x in terms:
        plain += x
    assert abs(plain - exact) > 2.3e-16 * exact     # the case is one a plain sum gets wrong


def test_rest_over_terrain_stays_at_rest():
    """A resting hydrostatic atmosphere over a hill stays exactly at rest (p' = 0, B = 0)."""
    wl = W.hill_bubble(nx=16, ny=16, nz=12, dx=300.0, dz0=120.0, ratio=1.02).with_(dtheta=None)
    o = make_oracle(wl)
    o.step(20)
    s = o.state()
    assert np.max(np.abs(s["rhow"])) <= 1e-12
    assert np.all(s["rhou"] == 0.0) and np.all(s["rhov"] == 0.0)


def test_buoyancy_sign_cold_sinks_warm_rises():
    """Reading R3: B = -(rho - rho0) g on the vertical component; the paper's density current
    descends (Sec. 4.1.1) and the warm bubble rises (Sec. 4.1.2)."""
    wl = W.density_current(nx=64, ny=1, nz=32, dx=200.0)
    o = make_oracle(wl)
    o.step(4)
    w = o.get("rhow")
    ic = wl.nx // 2
    k3 = int(3000.0 / 200.0)
    assert w[k3, 0, ic] < -0.01
    o = make_oracle(wl.with_(dtheta=-wl.dtheta))
    o.step(4)
    assert o.get("rhow")[k3, 0, ic] > 0.01


def test_no_substep_identity_when_acoustic_terms_are_off():
    """Reading R9: with every linear term of App. C switched off, the substep stage gives
    S^n + alpha_s dt R(S^t), i.e. the plain RK3 of Sec. 3.1."""
    wl = W.density_current(nx=32, ny=4, nz=16, dx=400.0, dt=0.1)
    a = make_oracle(wl, acoustic_off=1)
    b = make_oracle(wl, substep_mode=1)
    a.step(2); b.step(2)
    for k in ("rho", "rhotheta", "rhou", "rhov", "rhow"):
        x, y = a.get(k), b.get(k)
        scale = max(np.max(np.abs(y)), 1e-30)
        assert np.max(np.abs(x - y)) / scale < 1e-13, k


def _project(field, basis):
    return float(np.sum(field * basis) / np.sum(basis * basis))


def test_acoustic_standing_wave_frequency():
    """App. C linearised acoustics: with g = 0 a standing mode cos(kx) of 32 cells oscillates at
    omega = c k, c = sqrt(gamma p/rho) (continuous); the substepped discrete scheme stays
    within 0.5 %."""
    nx, dx = 32, 100.0
    wl = W.Workload("acoustic", nx, 1, 2, dx, dx, np.array([0.0, 100.0, 200.0]), dt=0.5,
                    n_substeps=6, gravity=0.0)
    o = make_oracle(wl)
    rho0 = o.get("rho"); rt0 = o.get("rhotheta")
    x = (np.arange(nx) + 0.5) * dx
    mode = np.cos(2 * np.pi * x / (nx * dx))[None, None, :] * np.ones((2, 1, 1))
    eps = 1e-5
    o.set("rhotheta", rt0 * (1 + eps * mode))
    o.set("rho", rho0 * (1 + eps / GAMMA * mode))
    ts, amps = [], []
    for n in range(60):
        amps.append(_project(o.get("rhotheta") - rt0, mode))
        ts.append(n * wl.dt)
        o.step(1)
    ts, amps = np.array(ts), np.array(amps)
    from scipy.optimize import curve_fit
    p0 = 1.0e5
    rho = rho0[0, 0, 0]
    c = np.sqrt(GAMMA * p0 / rho)
    k = 2 * np.pi / (nx * dx)
    f = lambda t, A, s, w, ph: A * np.exp(-s * t) * np.cos(w * t + ph)
    popt, _ = curve_fit(f, ts, amps, p0=[amps[0], 0.0, c * k, 0.0])
    assert abs(popt[2] / (c * k) - 1.0) < 5e-3


def test_gravity_wave_frequency():
    """Buoyancy oscillation of a mode sin(kx) sin(mz) between rigid lids in a stratified
    atmosphere (N = 0.01): omega = N k / sqrt(k^2 + m^2) within 2 %."""
    nx, nz, dx, dz = 20, 25, 500.0, 200.0
    zeta = np.arange(nz + 1) * dz
    wl = W.Workload("gw", nx, 1, nz, dx, dx, zeta, dt=2.0, n_substeps=6, brunt_N=0.01)
    x = (np.arange(nx) + 0.5) * dx
    zc = 0.5 * (zeta[1:] + zeta[:-1])
    kx, mz = 2 * np.pi / (nx * dx), np.pi / (nz * dz)
    mode = np.sin(mz * zc)[:, None, None] * np.sin(kx * x)[None, None, :]
    wl = wl.with_(dtheta=1e-3 * mode)
    o = make_oracle(wl)
    th0 = o.get("base_theta")
    ts, amps = [], []
    for n in range(700):
        if n % 5 == 0:
            th = o.get("rhotheta") / o.get("rho")
            amps.append(_project(th - th0, mode)); ts.append(n * wl.dt)
        o.step(1)
    from scipy.optimize import curve_fit
    w_exact = 0.01 * kx / np.sqrt(kx ** 2 + mz ** 2)
    f = lambda t, A, s, w, ph, B: A * np.exp(-s * t) * np.cos(w * t + ph) + B
    popt, _ = curve_fit(f, np.array(ts), np.array(amps), p0=[1e-3, 0.0, w_exact, 0.0, 0.0])
    assert abs(popt[2] / w_exact - 1.0) < 0.02


def test_inertial_oscillation_coriolis_sign():
    """f-plane forcing (Sec. 3.7): with g = 0 and u_g = v_g = 0 a uniform wind turns clockwise
    (northern hemisphere): u = U cos(f t), v = -U sin(f t)."""
    wl = W.Workload("cor", 8, 8, 2, 100.0, 100.0, np.array([0.0, 100.0, 200.0]), dt=10.0,
                    n_substeps=6, gravity=0.0, f_cor=1e-3)
    o = make_oracle(wl.with_(u=np.full((2, 8, 8), 10.0)))
    rho = o.get("rho")[0, 0, 0]
    o.step(50)
    t = 500.0
    u = o.get("rhou") / rho; v = o.get("rhov") / rho
    assert np.allclose(u, 10 * np.cos(1e-3 * t), atol=1e-6)
    assert np.allclose(v, -10 * np.sin(1e-3 * t), atol=1e-6)


def _uniform_box(nx, ny, nz, dx, dz, **kw):
    zeta = np.arange(nz + 1) * dz
    return W.Workload("box", nx, ny, nz, dx, dx, zeta, gravity=0.0, **kw)


def _rhs_with(o, rho, rt, ru, rv, rw):
    o.set("rho", rho); o.set("rhotheta", rt); o.set("rhou", ru); o.set("rhov", rv); o.set("rhow", rw)
    return o.slow_rhs()


def test_viscous_stress_divergence_discrete_eigenvalues():
    """Eq. stresstensor with constant nu: for u(y) = sin(2 pi y/L) the x-momentum tendency is
    rho nu lambda u with the 3-point eigenvalue lambda = -(4/dy^2) sin^2(pi dy/L); for u(x) the
    deviatoric 1/3 makes it (4/3) rho nu lambda u; heat: (rho nu/Pr_t) lambda theta'."""
    nx = ny = 16; nz = 3; dx = 50.0; nu = 7.5
    wl = _uniform_box(nx, ny, nz, dx, 50.0, closure=W.CLOSURE_CONST_NU, nu=nu, Pr_t=0.5)
    o1 = make_oracle(wl); o0 = make_oracle(wl.with_(closure=W.CLOSURE_NONE))
    rho = o1.get("rho"); rt = o1.get("rhotheta")
    r0 = rho[0, 0, 0]
    L = nx * dx
    lam = -(4.0 / dx ** 2) * np.sin(np.pi * dx / L) ** 2
    y = (np.arange(ny) + 0.5) * dx
    x_face = np.arange(nx) * dx
    zw = np.zeros((nz + 1, ny, nx))
    # u varies with y
    u = np.broadcast_to(np.sin(2 * np.pi * y / L)[None, :, None], rho.shape) * 0.01
    d = _rhs_with(o1, rho, rt, r0 * u, 0 * u, zw)["R_rhou"] - _rhs_with(o0, rho, rt, r0 * u, 0 * u, zw)["R_rhou"]
    np.testing.assert_allclose(d, r0 * nu * lam * u, atol=1e-15)
    # u varies with x (compressive: deviatoric 4/3)
    u = np.broadcast_to(np.sin(2 * np.pi * x_face / L)[None, None, :], rho.shape) * 0.01
    d = _rhs_with(o1, rho, rt, r0 * u, 0 * u, zw)["R_rhou"] - _rhs_with(o0, rho, rt, r0 * u, 0 * u, zw)["R_rhou"]
    np.testing.assert_allclose(d, (4.0 / 3.0) * r0 * nu * lam * u, atol=1e-15)
    # heat flux: theta(x) at cells
    xc = (np.arange(nx) + 0.5) * dx
    th = 300.0 + 0.1 * np.broadcast_to(np.sin(2 * np.pi * xc / L)[None, None, :], rho.shape)
    z = np.zeros_like(rho)
    d = _rhs_with(o1, rho, rho * th, z, z, zw)["R_rhotheta"] - _rhs_with(o0, rho, rho * th, z, z, zw)["R_rhotheta"]
    np.testing.assert_allclose(d, r0 * nu / 0.5 * lam * (th - 300.0), atol=1e-12)


def test_smagorinsky_linear_shear_closed_form():
    """Reading R6: u = S z gives |S| = S so mu_t = rho (Cs Delta)^2 S in the interior, and the
    resulting uniform stress has zero divergence there."""
    nx = ny = 8; nz = 10; dz = 20.0; dx = 40.0; S = 0.05
    wl = _uniform_box(nx, ny, nz, dx, dz, closure=W.CLOSURE_SMAGORINSKY, Cs=0.17)
    o = make_oracle(wl)
    rho = o.get("rho"); rt = o.get("rhotheta")
    zc = (np.arange(nz) + 0.5) * dz
    u = np.broadcast_to(S * zc[:, None, None], rho.shape)
    r = _rhs_with(o, rho, rt, rho * u, 0 * u, np.zeros((nz + 1, ny, nx)))
    mu = o.mu()
    Delta = (dx * dx * dz) ** (1.0 / 3.0)
    np.testing.assert_allclose(mu[1:-1], rho[1:-1] * (0.17 * Delta) ** 2 * S, rtol=1e-13)
    assert np.max(np.abs(r["R_rhou"][2:-2])) < 1e-15
    # Galilean invariance and the x<->y mirror: same mu for u + U and for v = S z
    r2 = _rhs_with(o, rho, rt, rho * (u + 3.0), 0 * u, np.zeros((nz + 1, ny, nx)))
    np.testing.assert_allclose(o.mu(), mu, rtol=1e-12)
    _rhs_with(o, rho, rt, 0 * u, rho * u, np.zeros((nz + 1, ny, nx)))
    np.testing.assert_allclose(o.mu(), mu, rtol=1e-13)


def _order_fit(ns, errs):
    return np.polyfit(np.log(ns), np.log(errs), 1)[0] * -1.0


@pytest.mark.parametrize("scheme,min_order", [(5, 4.8), (0, 4.0), (1, 4.5)])
def test_scalar_advection_operator_design_order(scheme, min_order):
    """Sec. 3.6: observed order of the theta flux divergence under uniform translation
    (linear upwind-5 -> 5; WENO5-JS/Z close to 5 on smooth data)."""
    errs, ns = [], [32, 64, 128]
    for nx in ns:
        dx = 6400.0 / nx
        wl = _uniform_box(nx, 1, 2, dx, 100.0, scal_adv=scheme)
        o = make_oracle(wl)
        rho = o.get("rho")
        xc = (np.arange(nx) + 0.5) * dx
        k = 2 * np.pi / 6400.0
        # theta given as cell averages of 300 + sin(kx)
        th = 300.0 + (np.cos(k * (xc - dx / 2)) - np.cos(k * (xc + dx / 2))) / (k * dx)
        th = np.broadcast_to(th[None, None, :], rho.shape)
        U = 5.0
        r = _rhs_with(o, rho, rho * th, rho * U, 0 * rho, np.zeros((3, 1, nx)))
        # exact cell-average tendency: -rho U d theta/dx averaged over the cell
        ex = -rho * U * (np.sin(k * (xc + dx / 2)) - np.sin(k * (xc - dx / 2)))[None, None, :] / dx
        errs.append(np.max(np.abs(r["R_rhotheta"] - ex)))
    assert _order_fit(ns, errs) > min_order


def test_momentum_advection_operator_design_order():
    """Upwind-5 momentum advection (Sec. 3.6, reading R5) of u(y) by a uniform v: order 5."""
    errs, ns = [], [32, 64, 128]
    for ny in ns:
        dy = 6400.0 / ny
        wl = _uniform_box(1, ny, 2, dy, 100.0)
        o = make_oracle(wl)
        rho = o.get("rho"); rt = o.get("rhotheta")
        k = 2 * np.pi / 6400.0
        yc = (np.arange(ny) + 0.5) * dy
        u = (np.cos(k * (yc - dy / 2)) - np.cos(k * (yc + dy / 2))) / (k * dy)
        u = np.broadcast_to(u[None, :, None], rho.shape)
        V = 3.0
        r = _rhs_with(o, rho, rt, rho * u, rho * V + 0 * u, np.zeros((3, ny, 1)))
        ex = -rho * V * ((np.sin(k * (yc + dy / 2)) - np.sin(k * (yc - dy / 2))) / dy)[None, :, None]
        errs.append(np.max(np.abs(r["R_rhou"] - ex)))
    assert _order_fit(ns, errs) > 4.8


def test_rk3_time_order():
    """Sec. 3.1: the RK3 scheme is third order in time (no-substep mode, smooth translation)."""
    nx, dx = 32, 200.0
    wl = _uniform_box(nx, 1, 2, dx, 100.0, scal_adv=5)
    xc = (np.arange(nx) + 0.5) * dx
    dth = np.broadcast_to((0.5 * np.sin(2 * np.pi * xc / (nx * dx)))[None, None, :], (2, 1, nx))
    T = 4.0
    sols = {}
    for n in (8, 16, 32, 128):
        o = make_oracle(wl.with_(dt=T / n, dtheta=dth, u=np.full((2, 1, nx), 20.0)), substep_mode=1)
        o.step(n)
        sols[n] = o.get("rho")
    e = [np.max(np.abs(sols[n] - sols[128])) for n in (8, 16, 32)]
    assert np.log2(e[0] / e[1]) > 2.6 and np.log2(e[1] / e[2]) > 2.6


def test_most_neutral_and_stability_function():
    """Reading R15: neutral u* = kappa U / ln(z1/z0); Businger-Dyer psi_m is the integral of
    (1 - phi_m)/zeta with phi_m = (1 - 16 zeta)^(-1/4) (unstable) and 1 + 5 zeta (stable)."""
    assert oracle.ustar(10.0, 5.0, 0.1) == pytest.approx(0.4 * 10.0 / np.log(50.0), rel=1e-15)
    from scipy.integrate import quad
    for z in (-3.0, -0.5, -0.01):
        ex = quad(lambda s: (1 - (1 - 16 * s) ** -0.25) / s, z, 0.0)[0] * -1.0
        assert oracle.psi_m(z) == pytest.approx(ex, rel=1e-7)
    for z in (0.2, 0.9):
        ex = -quad(lambda s: (5 * s) / s, 0.0, z)[0]
        assert oracle.psi_m(z) == pytest.approx(ex, rel=1e-12)
    # unstable surface flux raises u* above neutral
    assert oracle.ustar(5.0, 20.0, 0.1, Q=0.2) > oracle.ustar(5.0, 20.0, 0.1)


def test_most_surface_drag_decelerates():
    """MOST bottom stress removes momentum from the first level only, with rate rho u*^2/dz."""
    nx = ny = 4; nz = 4; dz = 10.0
    wl = _uniform_box(nx, ny, nz, 10.0, dz, surface=W.SURFACE_MOST, z0=0.1)
    o = make_oracle(wl)
    rho = o.get("rho"); rt = o.get("rhotheta")
    r = _rhs_with(o, rho, rt, rho * 8.0, 0 * rho, np.zeros((nz + 1, ny, nx)))
    us = 0.4 * 8.0 / np.log(5.0 / 0.1)
    np.testing.assert_allclose(r["R_rhou"][0], -rho[0] * us ** 2 / dz, rtol=1e-13)
    assert np.max(np.abs(r["R_rhou"][1:])) < 1e-13


def test_openmp_oracle_is_bitwise_serial():
    """The OpenMP loops of the oracle write disjoint elements; 1 and 4 threads agree bit for bit."""
    import subprocess, sys, json
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from conftest import make_oracle\n"
        "from paper_2412_04395_gb300 import workloads as W\n"
        "wl = W.hill_bubble(nx=20, ny=18, nz=12, dx=300.0, dz0=100.0, ratio=1.03, h0=300.0)\n"
        "o = make_oracle(wl); o.step(2); s = o.state()\n"
        "print(sum(hash(v.tobytes()) for v in s.values()))\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for n in (1, 4):
        env = dict(os.environ, OMP_NUM_THREADS=str(n), PYTHONHASHSEED="0")
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True).stdout.strip())
    assert outs[0] == outs[1] and outs[0] != ""


def test_most_surface_heat_flux_warms_the_lowest_cell():
    """Sec. 3.8: a positive (upward) kinematic surface heat flux Q heats the first level at rate
    rho Q / dz and leaves the levels above untouched."""
    nx = ny = 4; nz = 4; dz = 10.0; Q = 0.2
    wl = _uniform_box(nx, ny, nz, 10.0, dz, surface=W.SURFACE_MOST, z0=0.1, sfc_theta_flux=Q)
    o = make_oracle(wl)
    rho = o.get("rho"); rt = o.get("rhotheta")
    r = _rhs_with(o, rho, rt, 0 * rho, 0 * rho, np.zeros((nz + 1, ny, nx)))
    np.testing.assert_allclose(r["R_rhotheta"][0], rho[0] * Q / dz, rtol=1e-13)
    assert np.max(np.abs(r["R_rhotheta"][1:])) < 1e-13


def test_sullivan_coordinate_beta3_metrics_and_rest():
    """Sec. 3.4: z = zeta + (1 - zeta/z_t)^beta h with beta = 3 (Sullivan).  The cell heights are
    the closed form dzeta_k + (s_{k+1} - s_k) h_c, s = (1 - zeta/z_t)^3 and h_c the 4-node
    average of the nodal terrain; a resting hydrostatic atmosphere over the hill stays at rest."""
    wl = W.hill_bubble(nx=16, ny=16, nz=12, dx=300.0, dz0=120.0, ratio=1.02).with_(dtheta=None, terrain_beta=3)
    o = make_oracle(wl, init=False)
    zeta = np.asarray(wl.zeta)
    s = (1.0 - zeta / zeta[-1]) ** 3
    h = np.asarray(wl.terrain)
    hc = 0.25 * (h + np.roll(h, -1, axis=1) + np.roll(h, -1, axis=0) + np.roll(np.roll(h, -1, axis=0), -1, axis=1))
    expect = np.diff(zeta)[:, None, None] + np.diff(s)[:, None, None] * hc[None, :, :]
    assert np.allclose(o.geom("Hc"), expect, rtol=1e-13, atol=0)
    # beta = 3 flattens the coordinate surfaces faster with height than beta = 1
    s1 = 1.0 - zeta / zeta[-1]
    assert np.all(s[1:-1] < s1[1:-1])
    r = make_oracle(wl)
    r.step(20)
    st = r.state()
    assert np.max(np.abs(st["rhow"])) <= 1e-12
    assert np.all(st["rhou"] == 0.0) and np.all(st["rhov"] == 0.0)
