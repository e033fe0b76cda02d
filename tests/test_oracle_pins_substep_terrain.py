"""More oracle pins: conservation of every flux-form quantity, the linearised hydrostatic
balance inside an acoustic substep (App. C), terrain pressure-gradient cancellation and the
Omega metric (App. B), divergence damping, and advection order in every direction."""
import numpy as np
import pytest

import oracle
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

RD, CP = 287.0, 1004.5
CV = CP - RD
GAMMA = CP / CV
G = 9.81


def test_rhotheta_and_momentum_conserved():
    """Eq. theta is in flux form: sum(rho theta V) is conserved on a stratified periodic domain
    with walls; on flat terrain without Coriolis/surface drag total x-momentum is conserved."""
    wl = W.hill_bubble(nx=16, ny=16, nz=16, dx=250.0, dz0=100.0, ratio=1.03, h0=300.0)
    o = make_oracle(wl)
    o.set_initial(wl.dtheta, np.full(o.shape_c, 4.0), np.full(o.shape_c, -2.0), None)
    V = o.geom("Hc") * wl.dx * wl.dy
    t0 = np.sum(o.get("rhotheta") * V)
    o.step(4)
    assert abs(np.sum(o.get("rhotheta") * V) - t0) / t0 < 5e-14
    wl = W.density_current(nx=48, ny=4, nz=24, dx=250.0)
    o = make_oracle(wl)
    o.set_initial(wl.dtheta, np.full(o.shape_c, 3.0), None, None)
    Hx = o.geom("Hx")
    m0 = np.sum(o.get("rhou") * Hx)
    o.step(4)
    assert abs(np.sum(o.get("rhou") * Hx) - m0) / abs(m0) < 1e-13


def _column_state(nz=160, dz=25.0):
    zeta = np.arange(nz + 1) * dz
    wl = W.Workload("col", 4, 1, nz, 500.0, 500.0, zeta, dt=1.0, n_substeps=6, brunt_N=0.0)
    return wl


def test_substep_linear_hydrostatic_balance():
    """App. C, W'' row: with Theta'' and rho'' in linearised hydrostatic balance
    (d(gamma R_d pi Theta'')/dz = -g rho''), the vertical pressure-gradient, Theta''-buoyancy and
    rho''-buoyancy terms cancel, so one substep leaves W'' at truncation level - far below the
    size of the Theta''-buoyancy term alone (whose sign and factor R_d/c_v this pins)."""
    wl = _column_state()
    o = make_oracle(wl)
    rho0 = o.get("base_rho"); th0 = o.get("base_theta"); zc = o.geom("zc")
    pi0 = (o.get("base_p") / 1.0e5) ** (RD / CP)
    # wide enough that the O(dz^2) truncation of the two large terms stays well below the
    # Theta''-buoyancy term (ratio ~ g (R_d/c_v) L^2 / (theta c^2) >> (dz/L)^2)
    f = lambda z: np.exp(-((z - 2000.0) / 600.0) ** 2)
    eps = 1e-3
    Theta = eps * rho0 * th0 * f(zc)
    # rho'' = -(1/g) d/dz (gamma R_d pi0 Theta''), derivative of the smooth profile by a fine
    # centred difference in physical height
    h = 1e-2
    def C2T(z):
        pi_z = 1.0 - G * z / (CP * 300.0) * (1.0)  # neutral column: pi0 linear in z
        rt = (1.0e5 / RD) * pi_z ** (CV / RD)        # rho0 theta0 from the continuous HSE
        return GAMMA * RD * pi_z * eps * rt * f(z)
    rhoX = -(C2T(zc + h) - C2T(zc - h)) / (2 * h) / G
    X = {"rho": rhoX, "rhotheta": Theta, "rhou": np.zeros(o.shape_c), "rhov": np.zeros(o.shape_c),
         "rhow": np.zeros(o.shape_w)}
    dtau = 0.2
    out = o.substep_once(dtau, X)
    w = out["rhow"][1:-1, 0, 0]
    # size of the Theta''-buoyancy term alone at w-faces
    tb = dtau * G * rho0 * (RD / CV) * Theta / (rho0 * th0)
    tb = 0.5 * (tb[1:, 0, 0] + tb[:-1, 0, 0])
    assert np.max(np.abs(w)) < 0.1 * np.max(np.abs(tb))
    assert np.max(np.abs(out["rhou"])) == 0.0


def test_vertical_acoustic_standing_wave():
    """Vertically propagating sound between rigid lids (g = 0): mode cos(m z) in Theta'',
    omega = c m within 1 % (implicit vertical terms of App. C)."""
    nz, dz = 32, 50.0
    zeta = np.arange(nz + 1) * dz
    wl = W.Workload("vac", 2, 1, nz, 100.0, 100.0, zeta, dt=0.05, n_substeps=6, gravity=0.0)
    o = make_oracle(wl)
    rho0 = o.get("rho"); rt0 = o.get("rhotheta")
    zc = 0.5 * (zeta[1:] + zeta[:-1])
    m = np.pi / (nz * dz)
    mode = np.cos(m * zc)[:, None, None] * np.ones((1, 1, 2))
    o.set("rhotheta", rt0 * (1 + 1e-5 * mode)); o.set("rho", rho0 * (1 + 1e-5 / GAMMA * mode))
    ts, amps = [], []
    for n in range(200):
        amps.append(float(np.sum((o.get("rhotheta") - rt0) * mode) / np.sum(mode * mode))); ts.append(n * wl.dt)
        o.step(1)
    from scipy.optimize import curve_fit
    c = np.sqrt(GAMMA * 1.0e5 / rho0[0, 0, 0])
    fn = lambda t, A, s, w, ph: A * np.exp(-s * t) * np.cos(w * t + ph)
    popt, _ = curve_fit(fn, np.array(ts), np.array(amps), p0=[amps[0], 0.0, c * m, 0.0])
    assert abs(popt[2] / (c * m) - 1.0) < 1e-2


def test_divergence_damping_damps_horizontal_sound():
    """Sec. 3.1 / reading R10: forward-predicted pressure (beta_d > 0) damps a horizontal
    acoustic mode (8 cells per wavelength); beta_d = 0 leaves the forward-backward scheme
    neutral."""
    nx, dx = 8, 100.0
    ratio = {}
    for bd in (0.0, 0.1):
        wl = W.Workload("ac", nx, 1, 2, dx, dx, np.array([0.0, 100.0, 200.0]), dt=0.5,
                        n_substeps=6, gravity=0.0, beta_d=bd)
        o = make_oracle(wl)
        rho0 = o.get("rho"); rt0 = o.get("rhotheta")
        x = (np.arange(nx) + 0.5) * dx
        mode = np.cos(2 * np.pi * x / (nx * dx))[None, None, :] * np.ones((2, 1, 1))
        o.set("rhotheta", rt0 * (1 + 1e-5 * mode)); o.set("rho", rho0 * (1 + 1e-5 / GAMMA * mode))
        a0 = np.max(np.abs(o.get("rhotheta") - rt0))
        o.step(100)
        amp = []
        for n in range(12):          # > one period: envelope of the oscillation
            o.step(1)
            amp.append(np.max(np.abs(o.get("rhotheta") - rt0)))
        ratio[bd] = max(amp) / a0
    assert ratio[0.0] > 0.95 and ratio[0.0] < 1.0 + 1e-6
    assert ratio[0.1] < 0.5


def _terrain_case(nx=32, nz=20, dx=200.0, amp=150.0):
    x = np.arange(nx) * dx
    h = amp * (1.0 + np.sin(2 * np.pi * x / (nx * dx)))
    ter = np.tile(h, (2, 1))
    zeta = np.arange(nz + 1) * 200.0
    return W.Workload("ter", nx, 2, nz, dx, dx, zeta, terrain=ter, dt=0.5, n_substeps=6)


def test_terrain_pressure_gradient_cancels_on_height_surfaces():
    """App. B: p_x = p_xi - h_xi (p_zeta/h_zeta); for a pressure perturbation that depends on
    physical height only, the terrain correction cancels the along-coordinate derivative."""
    wl = _terrain_case()
    o = make_oracle(wl)
    rho0 = o.get("base_rho"); p0 = o.get("base_p"); zc = o.geom("zc")
    p = p0 + 200.0 * np.exp(-zc / 1500.0)
    rt = (1.0e5 / RD) * (p / 1.0e5) ** (1.0 / GAMMA)
    o.set("rho", rho0); o.set("rhotheta", rt)
    z = np.zeros(o.shape_c)
    o.set("rhou", z); o.set("rhov", z); o.set("rhow", np.zeros(o.shape_w))
    r = o.slow_rhs()
    pp = r["pp"]
    pxi = (pp - np.roll(pp, 1, axis=2)) / wl.dx
    interior = slice(1, wl.nz - 1)
    assert np.max(np.abs(r["R_rhou"][interior])) < 0.03 * np.max(np.abs(pxi[interior]))
    # the same cancellation in the acoustic substep's horizontal update (Theta'' form)
    X = {"rho": z, "rhotheta": 1e-3 * rt * np.exp(-zc / 1500.0), "rhou": z, "rhov": z,
         "rhow": np.zeros(o.shape_w)}
    out = o.substep_once(0.1, X)
    Txi = (X["rhotheta"] - np.roll(X["rhotheta"], 1, axis=2)) / wl.dx
    bound = 0.1 * GAMMA * RD * np.max(np.abs(Txi[interior]))
    assert np.max(np.abs(out["rhou"][interior])) < 0.05 * bound


def test_terrain_omega_free_stream_consistency():
    """App. B: with Omega = w - h_xi u (4-point averaged momenta) a uniform horizontal flow over
    terrain has nearly zero mass-flux divergence on interior levels (the vertical Omega flux
    balances the change of face height along x); a sign error leaves twice the imbalance."""
    wl = _terrain_case().with_(gravity=0.0)
    o = make_oracle(wl)
    rho = o.get("rho"); rt = o.get("rhotheta")
    U = 10.0
    o.set("rho", rho); o.set("rhotheta", rt); o.set("rhou", rho * U); o.set("rhov", 0 * rho)
    o.set("rhow", np.zeros(o.shape_w))
    r = o.slow_rhs()
    Hx = o.geom("Hx")
    dHx = (np.roll(Hx, -1, axis=2) - Hx) / wl.dx
    scale = np.max(np.abs(rho * U * dHx / o.geom("Hc"))[1:-1])
    assert np.max(np.abs(r["R_rho"][1:-1])) < 0.02 * scale


def test_weno5_reduces_to_upwind5_below_epsilon():
    """Reading R7 (eps = 1e-6): data whose smoothness indicators are far below eps give the
    linear weights, i.e. the upwind-5 interpolant."""
    rng = np.random.default_rng(5)
    for s in (1.0, -1.0):
        q = 300.0 + 1e-5 * rng.normal(size=6)
        lin = oracle.interp(q, s, 5)
        assert abs(oracle.weno5(q, s) - lin) < 1e-3 * np.ptp(q)


def _box(nx, ny, nz, dx, dz, **kw):
    zeta = np.arange(nz + 1) * dz
    return W.Workload("box", nx, ny, nz, dx, dx, zeta, gravity=0.0, **kw)


def _set(o, rho, rt, ru, rv, rw):
    o.set("rho", rho); o.set("rhotheta", rt); o.set("rhou", ru); o.set("rhov", rv); o.set("rhow", rw)
    return o.slow_rhs()


def _cellavg(k, x, d):
    return (np.cos(k * (x - d / 2)) - np.cos(k * (x + d / 2))) / (k * d)


def _dcellavg(k, x, d):
    return (np.sin(k * (x + d / 2)) - np.sin(k * (x - d / 2))) / d


@pytest.mark.parametrize("case", ["v_by_U", "w_by_U", "w_by_V", "u_by_W", "theta_by_V", "theta_by_W"])
def test_advection_order_each_direction(case):
    """Upwind-5 momentum / WENO5 scalar advection by a uniform velocity along every direction
    (x, y, z interior) converges at fifth order; catches shifted or transposed stencils."""
    errs, ns = [], [32, 64, 128]
    L = 6400.0
    k = 2 * np.pi / L
    for n in ns:
        d = L / n
        if case in ("v_by_U", "w_by_U"):
            wl = _box(n, 1, 12, d, 100.0); ax = 2
        elif case in ("w_by_V", "theta_by_V"):
            wl = _box(1, n, 12, d, 100.0); ax = 1
        else:
            wl = _box(1, 1, n, 100.0, d); ax = 0
        o = make_oracle(wl)
        rho = o.get("rho"); rt = o.get("rhotheta"); r0 = rho[0, 0, 0]
        shp_c, shp_w = o.shape_c, o.shape_w
        cen = (np.arange(n) + 0.5) * d
        fac = np.arange(n + (1 if ax == 0 else 0)) * d
        def along(v, shape):
            sh = [1, 1, 1]; sh[ax] = -1
            return np.broadcast_to(v.reshape(sh), shape)
        zc = np.zeros(shp_c); zw = np.zeros(shp_w)
        if case == "v_by_U":     # v at y-faces varying in x (cell-centred in x)
            v = along(_cellavg(k, cen, d), shp_c)
            r = _set(o, rho, rt, r0 * 4.0 + zc, r0 * v, zw); got, ex = r["R_rhov"], -r0 * 4.0 * along(_dcellavg(k, cen, d), shp_c)
        elif case == "w_by_U":   # w at w-faces varying in x; interior faces
            v = np.broadcast_to(_cellavg(k, cen, d)[None, None, :], shp_w).copy(); v[0] = 0; v[-1] = 0
            # faces 4..nz-4: vertical self-advection of the z-uniform w vanishes there
            r = _set(o, rho, rt, r0 * 4.0 + zc, zc, r0 * v); got = r["R_rhow"][4:-4]
            ex = -r0 * 4.0 * np.broadcast_to(_dcellavg(k, cen, d)[None, None, :], shp_w)[4:-4]
        elif case == "w_by_V":
            v = np.broadcast_to(_cellavg(k, cen, d)[None, :, None], shp_w).copy(); v[0] = 0; v[-1] = 0
            r = _set(o, rho, rt, zc, r0 * 4.0 + zc, r0 * v); got = r["R_rhow"][4:-4]
            ex = -r0 * 4.0 * np.broadcast_to(_dcellavg(k, cen, d)[None, :, None], shp_w)[4:-4]
        elif case == "u_by_W":   # u(z) advected by a uniform w (walls excluded: interior cells)
            u = along(_cellavg(k, cen, d), shp_c)
            ww = np.full(shp_w, r0 * 4.0); ww[0] = 0; ww[-1] = 0
            r = _set(o, rho, rt, r0 * u, zc, ww)
            got = r["R_rhou"][3:-4]; ex = (-r0 * 4.0 * along(_dcellavg(k, cen, d), shp_c))[3:-4]
        elif case == "theta_by_V":
            th = 300.0 + along(_cellavg(k, cen, d), shp_c)
            r = _set(o, rho, rho * th, zc, r0 * 4.0 + zc, zw); got = r["R_rhotheta"]
            ex = -r0 * 4.0 * along(_dcellavg(k, cen, d), shp_c)
        else:                    # theta(z) advected by uniform w, interior cells
            th = 300.0 + along(_cellavg(k, cen, d), shp_c)
            ww = np.full(shp_w, r0 * 4.0); ww[0] = 0; ww[-1] = 0
            r = _set(o, rho, rho * th, zc, zc, ww); got = r["R_rhotheta"][3:-4]
            ex = (-r0 * 4.0 * along(_dcellavg(k, cen, d), shp_c))[3:-4]
        errs.append(np.max(np.abs(got - ex)))
    order = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert order > (4.0 if case.startswith("theta") else 4.8), (case, errs)


def test_momentum_self_advection_second_order():
    """x-advection of u by u: the 2-point averaged advecting momentum (reading R5) makes the
    flux divergence second order; a shifted interpolation stencil drops it to first order."""
    errs, ns = [], [32, 64, 128]
    L = 6400.0; k = 2 * np.pi / L
    for n in ns:
        d = L / n
        wl = _box(n, 1, 2, d, 100.0)
        o = make_oracle(wl)
        rho = o.get("rho"); rt = o.get("rhotheta"); r0 = rho[0, 0, 0]
        xf = np.arange(n) * d
        u = np.broadcast_to((5.0 + np.sin(k * xf))[None, None, :], o.shape_c)
        r = _set(o, rho, rt, r0 * u, 0 * rho, np.zeros(o.shape_w))
        ex = -r0 * 2 * (5.0 + np.sin(k * xf)) * k * np.cos(k * xf)
        errs.append(np.max(np.abs(r["R_rhou"] - ex[None, None, :])))
    order = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert order > 1.8
