"""Pins of the oracle's learned-closure step (closure 3): the model's cell-centre stresses and heat
fluxes carried to edges and faces and differenced into the slow tendencies, checked against closed
forms that do not come from the oracle's code:

* a Fourier mode sin(k x) at cell centres, averaged to the faces or edges between two cells and
  differenced across a cell, has the exact discrete derivative k cos(k x) sin(k d)/(k d); a single
  difference across a face gives 2 sin(k d/2)/d cos(k x);
* the mean of two cells of a field linear in z is the value at the face between them (uniform
  spacing), and a quadratic's difference over a level spacing is exactly the sum of its two ends;
* zero stress and heat flux at the lid, and at the ground without MOST (slip walls);
* the Smagorinsky-Lilly fallback of a linear shear u = S z with theta = theta_s + G z is
  rho (Cs Delta)^2 S^2 in t13 and rho (Cs Delta)^2 S G / Pr_t in h3 (with the signs of
  down-gradient transport);
* a network whose outputs are exactly zero leaves the step bit for bit the no-closure step.
"""
import numpy as np
import pytest

from paper_2412_04395_gb300 import workloads as W
from conftest import make_oracle
from oracle import mlp_oracle as M

NX, NY, NZ, DX, DY, DZ = 24, 20, 12, 40.0, 50.0, 30.0


def _rest_oracle():
    wl = W.Workload("rest", NX, NY, NZ, DX, DY, W.uniform_zeta(NZ, DZ), closure=W.CLOSURE_LEARNED)
    return make_oracle(wl), make_oracle(wl.with_(closure=W.CLOSURE_NONE))


def _centres():
    x = (np.arange(NX) + 0.5) * DX
    y = (np.arange(NY) + 0.5) * DY
    zc = (np.arange(NZ) + 0.5) * DZ
    Z, Y, X = np.meshgrid(zc, y, x, indexing="ij")
    return X, Y, Z


def _diff_rhs(planes):
    """Slow tendencies with the model returning the given planes minus those without a closure."""
    o, o0 = _rest_oracle()
    o.set_sgs_model(lambda *state: planes)
    a, b = o.slow_rhs(), o0.slow_rhs()
    return {k: a[k] - b[k] for k in ("R_rho", "R_rhotheta", "R_rhou", "R_rhov", "R_rhow")}


def test_horizontal_fourier_modes_have_their_discrete_derivatives():
    X, Y, Z = _centres()
    kx, ky = 2 * np.pi / (NX * DX) * 3, 2 * np.pi / (NY * DY) * 2
    A = np.arange(1.0, 10.0)
    P = np.zeros((9, NZ, NY, NX))
    P[0] = A[0] * np.sin(kx * X)                            # t11
    P[1] = A[1] * np.sin(ky * Y)                            # t22
    P[3] = A[3] * (np.sin(ky * Y) + np.sin(kx * X))         # t12
    P[6] = A[6] * np.sin(kx * X)                            # h1
    P[7] = A[7] * np.cos(ky * Y)                            # h2
    d = _diff_rhs(P)
    xf, yf = X - 0.5 * DX, Y - 0.5 * DY                     # x-face and y-face positions
    # x-face of U: -(dt11/dx) across the face, -(dt12/dy) of the edge means around the face
    eu = -(A[0] * 2 * np.sin(kx * DX / 2) / DX * np.cos(kx * xf)
           + A[3] * np.cos(ky * Y) * np.sin(ky * DY) / DY)
    ev = -(A[1] * 2 * np.sin(ky * DY / 2) / DY * np.cos(ky * yf)
           + A[3] * np.cos(kx * X) * np.sin(kx * DX) / DX)
    et = -(A[6] * np.cos(kx * X) * np.sin(kx * DX) / DX - A[7] * np.sin(ky * Y) * np.sin(ky * DY) / DY)
    np.testing.assert_allclose(d["R_rhou"], eu, rtol=0, atol=1e-12 * np.max(np.abs(eu)))
    np.testing.assert_allclose(d["R_rhov"], ev, rtol=0, atol=1e-12 * np.max(np.abs(ev)))
    np.testing.assert_allclose(d["R_rhotheta"], et, rtol=0, atol=1e-12 * np.max(np.abs(et)))
    assert np.max(np.abs(d["R_rho"])) == 0.0
    assert np.max(np.abs(d["R_rhow"])) == 0.0


def test_vertical_profiles_and_the_walls():
    X, Y, Z = _centres()
    ky = 2 * np.pi / (NY * DY) * 2
    a4, a5, a2, a8 = 2.0, 3.0, 0.5, 7.0
    P = np.zeros((9, NZ, NY, NX))
    P[4] = a4 * Z                                           # t13 linear in z
    P[5] = a5 * np.cos(ky * Y)                              # t23 constant in z
    P[2] = a2 * Z ** 2                                      # t33 quadratic in z
    P[8] = a8 * Z                                           # h3 linear in z
    d = _diff_rhs(P)
    k = np.arange(NZ)[:, None, None]
    top = k == NZ - 1
    # t13 at interior xz-edges = a4 z_w(k) (zero at both walls): -1 a4 in every cell but the top
    # one, where only the edge below remains
    eu = np.where(top, a4 * (NZ - 1), -a4) * np.ones((NZ, NY, NX))
    np.testing.assert_allclose(d["R_rhou"], eu, rtol=0, atol=1e-12 * a4 * NZ)
    # t23 = a5 cos(ky y) cos(ky dy/2) at interior yz-edges: only the two wall cells see a jump
    yf = Y - 0.5 * DY
    e23 = a5 * np.cos(ky * yf) * np.cos(ky * DY / 2)
    ev = np.zeros((NZ, NY, NX))
    ev[0] = -e23[0] / DZ
    ev[-1] = e23[-1] / DZ
    np.testing.assert_allclose(d["R_rhov"], ev, rtol=0, atol=1e-12 * a5)
    # W at interior w-faces: -(t33(k) - t33(k-1))/dz = -2 a2 z_w(k), and -d(t23)/dy of the edges
    zw = np.arange(1, NZ) * DZ
    ew = -2 * a2 * zw[:, None, None] + a5 * np.sin(ky * Y[1:]) * np.sin(ky * DY) / DY
    np.testing.assert_allclose(d["R_rhow"][1:NZ], ew, rtol=0, atol=1e-12 * a2 * NZ * DZ)
    assert np.max(np.abs(d["R_rhow"][0])) == 0.0 and np.max(np.abs(d["R_rhow"][NZ])) == 0.0
    # h3 linear: -a8 in every cell but the top one (no flux through the lid or the slip ground)
    et = np.where(top, a8 * (NZ - 1), -a8) * np.ones((NZ, NY, NX))
    np.testing.assert_allclose(d["R_rhotheta"], et, rtol=0, atol=1e-12 * a8 * NZ)


def _shear_state(S, G, th_s=300.0):
    zc = (np.arange(NZ) + 0.5) * DZ
    rho = np.full((NZ, NY, NX), 1.1)
    rt = rho * (th_s + G * zc)[:, None, None]
    ru = rho * (S * zc)[:, None, None] * np.ones((NZ, NY, NX))
    return rho, rt, ru, np.zeros((NZ, NY, NX)), np.zeros((NZ + 1, NY, NX))


def _net(seed, in_sd, out_mu=None, out_sd=None, zero=False):
    rng = np.random.default_rng(seed)
    p = []
    for a, b in zip(M.LAYERS[:-1], M.LAYERS[1:]):
        Wt = np.zeros((b, a)) if zero else rng.standard_normal((b, a)) / np.sqrt(a)
        p.append((Wt, np.zeros(b) if zero else 0.1 * rng.standard_normal(b)))
    return M.pack_blob(p, np.zeros(12), np.full(12, in_sd),
                       np.zeros(9) if out_mu is None else out_mu, np.ones(9) if out_sd is None else out_sd)


def test_fallback_is_smagorinsky_lilly_of_a_linear_shear():
    S, G, Cs, Pr = 0.02, 0.003, 0.17, 1.0 / 3.0
    zeta = W.uniform_zeta(NZ, DZ)
    th0 = 300.0 + G * (np.arange(NZ) + 0.5) * DZ
    # every standardised input far beyond |z| = 6: every cell falls back
    m = M.LearnedClosure(_net(3, in_sd=1e-9), zeta, DX, DY, th0, Cs, Pr)
    with np.errstate(over="ignore"):   # the network's own outputs overflow; they are not used
        P = m(*_shear_state(S, G))
    assert m.fallbacks == [NX * NY * NZ]
    d2 = (Cs * np.cbrt(DX * DY * DZ)) ** 2
    np.testing.assert_allclose(P[4], -1.1 * d2 * S * S, rtol=1e-13)
    # theta = rho theta / rho differenced across a level: cancellation of 300 K against 0.09 K
    np.testing.assert_allclose(P[8], -1.1 * d2 * S * G / Pr, rtol=1e-11)
    for q in (0, 1, 2, 3, 5, 6, 7):
        assert np.max(np.abs(P[q])) <= 1e-13 * d2 * S * S, q


def test_network_cells_take_the_network_and_keep_the_density_weight():
    """Inputs well inside |z| <= 6: no cell falls back, and each plane is rho times the network's
    de-standardised output (here a network of zero weights: out_mu + out_sd b4 = out_mu)."""
    S, G = 0.02, 0.003
    zeta = W.uniform_zeta(NZ, DZ)
    th0 = 300.0 + G * (np.arange(NZ) + 0.5) * DZ
    omu = np.linspace(-0.3, 0.5, 9)
    omu[:6] = [0.01, 0.02, -0.03, 0.0, 0.0, 0.0]   # zero S11..S33, S12, S23: no backscatter limit applies
    m = M.LearnedClosure(_net(4, in_sd=1e3, out_mu=omu, zero=True), zeta, DX, DY, th0, 0.17, 1.0 / 3.0)
    P = m(*_shear_state(S, G))
    assert m.fallbacks == [0] and m.margin > 5.0
    omu32 = omu.astype(np.float32).astype(np.float64)   # the blob carries FP32 statistics
    for q in range(9):
        np.testing.assert_array_equal(P[q], 1.1 * omu32[q])


def test_zero_network_step_is_the_no_closure_step():
    wl = W.convective_abl(nx=16, ny=12, nz=20, dx=40.0).with_(precision=W.PREC_FP64)
    a = make_oracle(wl.with_(closure=W.CLOSURE_LEARNED))
    b = make_oracle(wl.with_(closure=W.CLOSURE_NONE))
    th0 = a.get("base_theta")[:, 0, 0]
    m = M.LearnedClosure(_net(5, in_sd=1e6, zero=True, out_sd=np.zeros(9)), wl.zeta, wl.dx, wl.dy, th0,
                         wl.Cs, wl.Pr_t)
    a.set_sgs_model(m)
    a.step(2)
    b.step(2)
    assert m.fallbacks == [0] * 6
    sa, sb = a.state(), b.state()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f


def test_learned_closure_without_a_model_is_refused():
    o, _ = _rest_oracle()
    with pytest.raises(AssertionError):
        o.step(1)


def test_backscatter_limit_inside_the_model_closed_form():
    """A network that returns a constant t13 = c > 0 on the linear shear u = S z (S13 = S/2): its
    transfer -2 c S13 is backscatter below -1/2 of Smagorinsky's 4 nu S13^2 (nu = (Cs Delta)^2 S),
    so t13 is scaled onto the bound: c (nu S13 / c) = (Cs Delta)^2 S^2 / 2, times rho."""
    S, G, Cs = 0.02, 0.003, 0.17
    zeta = W.uniform_zeta(NZ, DZ)
    th0 = 300.0 + G * (np.arange(NZ) + 0.5) * DZ
    omu = np.zeros(9)
    omu[4] = 0.05
    m = M.LearnedClosure(_net(6, in_sd=1e3, out_mu=omu, zero=True), zeta, DX, DY, th0, Cs, 1.0 / 3.0)
    P = m(*_shear_state(S, G))
    assert m.fallbacks == [0]
    d2 = (Cs * np.cbrt(DX * DY * DZ)) ** 2
    np.testing.assert_allclose(P[4], 1.1 * d2 * S * S / 2, rtol=1e-12)
