"""Pins of the oracle's moist dynamics and Kessler microphysics (Sec. 2.1 Eqs. nonprecip/precip and
the moist EOS, Sec. 2.4, App. C's moisture factors) and of its lateral relaxation zones (the open
boundaries of Sec. 3.8 / Table D).

Fixed by something other than the oracle's own formulas:
  * Klemp & Wilhelmson (1978) print the rain terminal velocity and the rain evaporation rate in cgs
    units (rho in g/cm^3, p in mb, V in cm/s): the oracle's SI forms must equal them;
  * Tetens' vapour pressure is 610.78 Pa at 273.16 K by construction and within 0.5% of the
    standard 2339 Pa at 20 C;
  * the moist EOS obeys Dalton's law: p = rho_d R_d T + rho_v R_v T with T = theta pi;
  * the moist base state is hydrostatic in its total density;
  * a saturation adjustment conserves q_v + q_c + q_r exactly and theta - L_v/(c_p pi) (q_c + q_r),
    and leaves a supersaturation far below the initial one; subsaturated air without condensate
    is left alone bit for bit; cloud water evaporates into subsaturated air;
  * autoconversion starts at q_c = 1e-3: below it no rain forms; above it one step makes
    dt k1 (q_c - 1e-3) of rain in saturated air;
  * rain falling through saturated air conserves rain + surface accumulation;
  * moist code without water is the dry code bit for bit; a moist atmosphere at rest stays at rest;
  * the relaxation zones leave the reference state alone and act only within their width.
"""
import numpy as np
import pytest

import oracle
from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle

RD, RV, CP, LV = 287.0, 461.5, 1004.5, 2.5e6


def test_rain_speed_matches_the_cgs_formula():
    for rho, qr, rs in ((1.1, 1e-3, 1.2), (0.6, 4e-3, 1.15), (1.0, 1e-5, 1.0)):
        rho_g = rho * 1e-3
        v_cgs = 3634.0 * (rho_g * qr) ** 0.1346 * (rs / rho) ** 0.5
        assert abs(oracle.rain_speed(rho, qr, rs) - v_cgs / 100.0) <= 1e-13 * v_cgs / 100.0
    assert oracle.rain_speed(1.0, 0.0, 1.0) == 0.0


def test_rain_evaporation_matches_the_cgs_formula():
    for rho, qv, qr, qvs, p in ((1.1, 0.008, 1e-3, 0.012, 9.0e4), (0.8, 0.002, 3e-3, 0.006, 6.0e4)):
        rg, pmb = rho * 1e-3, p / 100.0
        C = 1.6 + 124.9 * (rg * qr) ** 0.2046
        want = (1.0 / rg) * (1.0 - qv / qvs) * C * (rg * qr) ** 0.525 / (5.4e5 + 2.55e6 / (pmb * qvs))
        assert abs(oracle.rain_evap(rho, qv, qr, qvs, p) - want) <= 1e-13 * want
    assert oracle.rain_evap(1.0, 0.012, 1e-3, 0.010, 9e4) == 0.0          # supersaturated: none


def test_tetens_saturation():
    eps = RD / RV
    es0 = 610.78
    q = oracle.qvs(273.16, 1.0e5)
    assert abs(q - eps * es0 / (1.0e5 - es0)) <= 1e-15
    q20 = oracle.qvs(293.15, 1.0e5)
    es20 = q20 * 1.0e5 / (eps + q20)
    assert abs(es20 - 2339.0) < 0.005 * 2339.0


def moist_column(nx=4, ny=4, nz=30, dz=100.0, **kw):
    zeta = W.uniform_zeta(nz, dz)
    top = nz * dz
    base = dict(dt=1.0, n_substeps=6, moist=1,
                knots=(np.array([0.0, top]), np.array([300.0, 300.0 + 0.004 * top])),
                qv_knots=(np.array([0.0, top]), np.array([0.012, 0.004])))
    base.update(kw)
    return W.Workload("moist", nx, ny, nz, dz, dz, zeta, **base)


def _T_p(o):
    """temperature and pressure of the oracle's current state (moist EOS)"""
    r = o.slow_rhs()
    p = r["pp"] + o.get("base_p")
    return r["theta"] * r["pi"], p, r["pi"]


def test_moist_eos_obeys_daltons_law_and_the_base_state_is_hydrostatic():
    wl = moist_column(nz=40)
    o = make_oracle(wl)
    T, p, _ = _T_p(o)
    rho, rqv = o.get("rho"), o.get("rhoqv")
    np.testing.assert_allclose(p, rho * RD * T + rqv * RV * T, rtol=1e-13)
    # total-density hydrostatic residual between levels: p_k - p_{k-1} + g dz (rho_k + rho_{k-1})/2
    p0, r0 = o.get("base_p")[:, 0, 0], o.get("base_rho")[:, 0, 0]
    res = p0[1:] - p0[:-1] + 9.81 * 100.0 * 0.5 * (r0[1:] + r0[:-1])
    assert np.abs(res).max() <= 1e-9 * p0.max()
    # the base state's total density is its dry density times 1 + q_v0
    qv0 = o.get("base_qv")
    np.testing.assert_allclose(o.get("rho") * (1 + qv0), o.get("base_rho"), rtol=1e-14)


def _supersaturated(o, factor):
    """Sets q_v = factor x q_vs at every cell.  The vapour enters the EOS (at fixed rho theta,
    more vapour means a higher pressure and temperature), so q_v is iterated to the fixed point
    q_v = factor q_vs(T(q_v), p(q_v)); returns that q_vs."""
    rho = o.get("rho")
    for _ in range(40):
        T, p, _ = _T_p(o)
        qvs = np.vectorize(oracle.qvs)(T, p)
        o.set("rhoqv", rho * qvs * factor)
    return qvs


def test_saturation_adjustment_conserves_water_and_liquid_theta():
    wl = moist_column()
    o = make_oracle(wl)
    qvs0 = _supersaturated(o, 1.05)
    rho = o.get("rho")
    o.set("rhoqc", rho * 2e-4)                   # a little cloud, below the autoconversion threshold
    _, p0, pie = _T_p(o)
    qt0 = (o.get("rhoqv") + o.get("rhoqc") + o.get("rhoqr")) / rho
    thl0 = o.get("rhotheta") / rho - LV / (CP * pie) * (o.get("rhoqc") + o.get("rhoqr")) / rho
    s0 = o.get("rhoqv") / rho - qvs0
    o.kessler()
    qt1 = (o.get("rhoqv") + o.get("rhoqc") + o.get("rhoqr")) / rho
    thl1 = o.get("rhotheta") / rho - LV / (CP * pie) * (o.get("rhoqc") + o.get("rhoqr")) / rho
    np.testing.assert_allclose(qt1, qt0, rtol=1e-14)
    np.testing.assert_allclose(thl1, thl0, rtol=1e-14)
    assert np.all(o.get("rhoqc") / rho > 2e-4)   # vapour condensed
    # the adjustment is isobaric (pressure and Exner function of the state before it).  At that
    # pressure and the new temperature the remaining supersaturation is the linearisation's: the
    # standard one-step form takes dq_vs/dT = q_vs 4098.17/(T - 35.86)^2, which leaves out the
    # factor p / (p - e_s) of q_vs = eps e_s / (p - e_s) (1 + e_s/p, up to ~4% near the ground),
    # so a few per cent of the initial supersaturation is left, of the opposite sign
    T1 = o.get("rhotheta") / rho * pie
    s1 = o.get("rhoqv") / rho - np.vectorize(oracle.qvs)(T1, p0)
    es_over_p = np.vectorize(oracle.qvs)(T1, p0) / (RD / RV)
    assert np.all(np.abs(s1) <= 1.5 * es_over_p * np.abs(s0) + 1e-9)
    assert np.all(s1 <= 0.0)


def test_subsaturated_air_without_condensate_is_left_alone():
    wl = moist_column()
    o = make_oracle(wl)
    before = o.state()
    o.kessler()
    after = o.state()
    for k in before:
        assert np.array_equal(before[k], after[k]), k


def test_cloud_evaporates_into_subsaturated_air():
    wl = moist_column()
    o = make_oracle(wl)
    rho = o.get("rho")
    o.set("rhoqc", rho * 1e-5)                  # too little cloud to saturate the air
    th0 = o.get("rhotheta") / rho
    o.kessler()
    assert np.all(o.get("rhoqc") == 0.0)
    assert np.all(o.get("rhotheta") / rho < th0)   # evaporative cooling


def test_autoconversion_threshold_and_rate():
    wl = moist_column()
    for qc, want_rain in ((0.9e-3, 0.0), (2.0e-3, 1.0 * 1e-3 * (2.0e-3 - 1e-3))):
        o = make_oracle(wl)
        _supersaturated(o, 1.0)                  # exactly saturated: no adjustment
        rho = o.get("rho")
        o.set("rhoqc", rho * qc)
        o.kessler()
        qr = o.get("rhoqr") / rho
        np.testing.assert_allclose(qr, want_rain, rtol=1e-9, atol=1e-18)


def test_falling_rain_budget_closes_with_the_surface_accumulation():
    wl = moist_column(nz=30, dt=2.0)
    o = make_oracle(wl)
    _supersaturated(o, 1.0)
    rho = o.get("rho")
    qr = np.zeros(rho.shape)
    qr[5:12] = 2e-3
    o.set("rhoqr", rho * qr)
    H = o.geom("Hc")
    total0 = float(np.sum(o.get("rhoqr") * H))
    for _ in range(40):
        o.kessler()
    rain = float(np.sum(o.get("rhoqr") * H))
    fallen = float(np.sum(o.precip())) * 1000.0          # kg per m^2 of column, summed
    assert fallen > 0.0
    assert abs(rain + fallen - total0) <= 1e-12 * total0
    # the rain has moved down: its centre of mass is lower
    zc = o.geom("zc")
    assert np.sum(o.get("rhoqr") * H * zc) / rain < np.sum(rho * qr * H * zc) / total0


def test_moist_code_without_water_is_the_dry_code():
    dry = W.density_current(nx=48, ny=3, nz=20, dx=400.0)
    moist = dry.with_(moist=1, qv_knots=(np.array([0.0, 1e5]), np.array([0.0, 0.0])))
    a, b = make_oracle(dry), make_oracle(moist)
    a.step(3)
    b.step(3)
    for f in ("rho", "rhotheta", "rhou", "rhov", "rhow"):
        assert np.array_equal(a.get(f), b.get(f)), f
    assert np.all(b.get("rhoqv") == 0.0)


def test_moist_atmosphere_at_rest_stays_at_rest():
    wl = moist_column(nx=6, ny=5, nz=40)
    o = make_oracle(wl)
    o.step(20)
    rho = o.get("rho")
    rw = o.get("rhow")
    assert np.abs(rw).max() / rho.min() < 1e-10
    assert np.abs(o.get("rhou")).max() < 1e-10


def test_relaxation_zones():
    wl = W.squall_line(nx=64, ny=3, nz=20, dx=500.0, dt=1.0, relax_width=5000.0, relax_tau=0.02)
    o = make_oracle(wl)
    on = o.slow_rhs()
    off = make_oracle(wl.with_(relax_tau=0.0)).slow_rhs()
    for k in on:
        assert np.array_equal(on[k], off[k]), k          # the reference state is not relaxed
    # a perturbation: relaxed inside the zones (10 cells at each edge) and nowhere else
    rt = o.get("rhotheta")
    rt2 = rt * (1.0 + 1e-3)
    o.set("rhotheta", rt2)
    p = make_oracle(wl.with_(relax_tau=0.0))
    p.set("rhotheta", rt2)
    d = o.slow_rhs()["R_rhotheta"] - p.slow_rhs()["R_rhotheta"]
    xc = (np.arange(64) + 0.5) * 500.0
    inside = (xc < 5000.0) | (xc > 64 * 500.0 - 5000.0)
    assert np.all(d[:, :, ~inside] == 0.0)
    assert np.all(d[:, :, inside] < 0.0)                  # back toward the reference
    rate = -d[0, 0] / (rt2 - rt)[0, 0]
    assert abs(rate[0] - 0.02) < 0.02 * 0.05             # near the full rate at the edge cell


def _uniform_vapour_case(Q=0.012):
    wl = moist_column(nx=16, ny=4, nz=12)
    X, Y, Z = W.cell_coords(16, 4, wl.zeta, wl.dx, wl.dy)
    return wl.with_(dtheta=0.5 * np.sin(2 * np.pi * X / 1600.0) * np.cos(np.pi * Z / 1200.0),
                    qv=np.full((12, 4, 16), Q)), Q


def test_moist_momentum_terms_carry_one_over_one_plus_qv_plus_qc():
    """Eq. mom: at rest (no advection) R_U = -(dp'/dx) / (1 + q_v + q_c) and
    R_W = (-(dp'/dz) + B) / (1 + q_v + q_c), B = -g (rho_m - rho0) with the total density
    rho_m = rho_d (1 + q_v + q_c + q_r), face means of the two cells."""
    wl, Q = _uniform_vapour_case()
    o = make_oracle(wl)
    # a pressure perturbation (the initial state is built at unchanged pressure)
    X, Y, Z = W.cell_coords(16, 4, wl.zeta, wl.dx, wl.dy)
    o.set("rhotheta", o.get("rhotheta") * (1.0 + 1e-4 * np.cos(2 * np.pi * X / 1600.0)))
    r = o.slow_rhs()
    pp = r["pp"]
    gx = -(pp - np.roll(pp, 1, axis=2)) / wl.dx
    assert np.abs(gx).max() > 1e-3
    np.testing.assert_allclose(r["R_rhou"], gx / (1 + Q), rtol=1e-12, atol=1e-14)
    rho, rho0 = o.get("rho"), o.get("base_rho")
    Bc = -9.81 * (rho * (1 + Q) - rho0)
    dz = wl.zeta[1] - wl.zeta[0]
    want = (-(pp[1:] - pp[:-1]) / dz + 0.5 * (Bc[1:] + Bc[:-1])) / (1 + Q)
    np.testing.assert_allclose(r["R_rhow"][1:-1], want, rtol=1e-10, atol=1e-12)


def test_substep_pressure_term_carries_one_over_one_plus_qv_plus_qc():
    """App. C: Delta U'' = -dtau gamma R_d pi^t / (1 + q_v^t + q_c^t) dTheta''/dxi.  A dry stage
    state and a moist one with the same pressure (hence the same pi: rho theta scaled by
    1 / (1 + (R_v/R_d) Q)) give U'' responses to the same Theta'' in the ratio 1 / (1 + Q)."""
    wl, Q = _uniform_vapour_case()
    dry = make_oracle(wl.with_(moist=0, qv=None, qv_knots=None))
    mst = make_oracle(wl)
    rho, rt = dry.get("rho"), dry.get("rhotheta")
    mst.set("rho", rho)
    mst.set("rhotheta", rt / (1.0 + (RV / RD) * Q))
    mst.set("rhoqv", rho * Q)
    np.testing.assert_allclose(mst.slow_rhs()["pi"], dry.slow_rhs()["pi"], rtol=1e-14)
    X, Y, Z = W.cell_coords(16, 4, wl.zeta, wl.dx, wl.dy)
    Xin = {k: np.zeros(dry.shape_w if k == "rhow" else dry.shape_c) for k in FIELDS5}
    Xin["rhotheta"] = 1e-3 * np.sin(2 * np.pi * X / 1600.0)
    ud = dry.substep_once(0.1, Xin)["rhou"]
    um = mst.substep_once(0.1, Xin)["rhou"]
    assert np.abs(ud).max() > 0
    np.testing.assert_allclose(um, ud / (1.0 + Q), rtol=1e-12, atol=1e-15 * np.abs(ud).max())


FIELDS5 = ("rho", "rhotheta", "rhou", "rhov", "rhow")
