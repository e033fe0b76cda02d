"""Pins of the learned-closure oracle (oracle/mlp_oracle.py): gradients against central finite
differences, closed forms of SiLU and of one Adam step, the Favre box filter on fields with known
moments, and second-order convergence of the closure features."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _params(seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    p = []
    for a, b in zip(M.LAYERS[:-1], M.LAYERS[1:]):
        p.append((rng.normal(size=(b, a)) * scale / np.sqrt(a), rng.normal(size=b) * 0.1))
    return p


def test_silu_closed_forms():
    assert M.silu(np.array(0.0)) == 0.0
    assert M.dsilu(np.array(0.0)) == pytest.approx(0.5, abs=1e-16)
    x = np.linspace(-6, 6, 41)
    h = 1e-6
    np.testing.assert_allclose(M.dsilu(x), (M.silu(x + h) - M.silu(x - h)) / (2 * h), rtol=1e-8, atol=1e-10)
    assert M.silu(np.array(40.0)) == pytest.approx(40.0, rel=1e-15)


def test_backprop_matches_finite_differences():
    p = _params(1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(7, 12))
    T = rng.normal(size=(7, 9))
    Y, cache = M.forward(p, X)
    loss, dY = M.mse(Y, T)
    g = M.backward(p, cache, dY)
    h = 1e-6
    for l in range(4):
        W, b = p[l]
        for (r, c) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, W.shape[1] // 3)]:
            Wp = W.copy(); Wp[r, c] += h
            Wm = W.copy(); Wm[r, c] -= h
            pp = list(p); pp[l] = (Wp, b)
            pm = list(p); pm[l] = (Wm, b)
            fd = (M.mse(M.forward(pp, X)[0], T)[0] - M.mse(M.forward(pm, X)[0], T)[0]) / (2 * h)
            assert g[l][0][r, c] == pytest.approx(fd, rel=1e-6, abs=1e-10)
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        pp = list(p); pp[l] = (W, bp)
        pm = list(p); pm[l] = (W, bm)
        fd = (M.mse(M.forward(pp, X)[0], T)[0] - M.mse(M.forward(pm, X)[0], T)[0]) / (2 * h)
        assert g[l][1][1] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_forward_with_zero_hidden_weights_is_a_closed_form():
    p = _params(3)
    p = [(np.zeros_like(W), b) if l < 3 else (W, b) for l, (W, b) in enumerate(p)]
    X = np.random.default_rng(4).normal(size=(5, 12))
    Y, _ = M.forward(p, X)
    hidden = M.silu(p[2][1])   # last hidden layer sees silu of its bias only
    np.testing.assert_allclose(Y, np.broadcast_to(p[3][0] @ hidden + p[3][1], Y.shape), rtol=1e-14)


def test_first_adam_step_closed_form():
    """Kingma & Ba: from zero moments the bias-corrected first step is -lr g/(|g| + eps)."""
    p = _params(5)
    g = [(np.full_like(W, 0.3), np.full_like(b, -2.0)) for W, b in p]
    m, v = M.adam_init(p)
    new, m1, v1 = M.adam_step(p, g, m, v, 1, lr=1e-3)
    for (W, b), (W1, b1) in zip(p, new):
        np.testing.assert_allclose(W1 - W, -1e-3 * 0.3 / (0.3 + 1e-8), rtol=1e-12)
        np.testing.assert_allclose(b1 - b, 1e-3 * 2.0 / (2.0 + 1e-8), rtol=1e-12)


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(6)
    X = rng.normal(size=(2048, 12))
    A = rng.normal(size=(12, 9)) * 0.3
    T = np.tanh(X @ A)
    p, losses = M.train(_params(7), X, T, epochs=20, batch=256, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0]


def _periodic_state(nx, ny, nz, fu=None, fv=None, fw=None, fth=None, rho=1.2):
    shape = (nz, ny, nx)
    r = np.full(shape, rho)
    ru = np.zeros(shape) if fu is None else rho * fu
    rv = np.zeros(shape) if fv is None else rho * fv
    rw = np.zeros((nz + 1, ny, nx)) if fw is None else rho * fw
    th = np.full(shape, 300.0) if fth is None else fth
    return r, r * th, ru, rv, rw


def test_box_filter_constant_and_linear_fields():
    """Constant fields filter to themselves with zero SGS terms; u linear in x over a block of r
    cells of width h gives t_11 = a^2 h^2 (r^2 - 1)/12 (the variance of r equispaced points)."""
    nx, ny, nz, h, a = 16, 8, 8, 10.0, 0.02
    st = _periodic_state(nx, ny, nz, fu=np.full((nz, ny, nx), 3.0))
    (rb, Rt, Ru, Rv, Rw), T = M.box_filter(*st, r=4)
    np.testing.assert_allclose(rb, 1.2); np.testing.assert_allclose(Ru, 3.6)
    assert np.max(np.abs(T)) < 1e-14 * 3.0 * 300.0 * 4   # round-off of <rho u theta>/rho - u theta (~900)
    # u at x-faces x = i h: u = a i h -> cell centres (i + 1/2) a h, block variance a^2 h^2 (16 - 1)/12
    xf = np.arange(nx) * h
    u = np.broadcast_to(a * xf, (nz, ny, nx)).copy()
    # keep the periodic seam outside the tested block: test blocks that do not touch the seam
    st = _periodic_state(nx, ny, nz, fu=u)
    (_, _, _, _, _), T = M.box_filter(*st, r=4)
    np.testing.assert_allclose(T[:, :, :3, 0], a * a * h * h * 15.0 / 12.0, rtol=1e-12)
    np.testing.assert_allclose(T[:, :, :3, 1:6], 0.0, atol=1e-14)
    np.testing.assert_allclose(T[:, :, :3, 6:], 0.0, atol=1e-15 * 300.0 * 4)   # u theta round-off


def test_box_filter_heat_flux_of_correlated_fields():
    """theta' = c u' inside each block gives h_1 = c t_11 (u and theta perfectly correlated)."""
    nx, ny, nz = 8, 4, 4
    rng = np.random.default_rng(8)
    u = rng.normal(size=(nz, ny, nx))
    uf = u.copy()
    uc = 0.5 * (uf + np.roll(uf, -1, axis=2))
    th = 300.0 + 0.7 * uc
    st = _periodic_state(nx, ny, nz, fu=uf, fth=th)
    _, T = M.box_filter(*st, r=4)
    np.testing.assert_allclose(T[..., 6], 0.7 * T[..., 0], rtol=1e-10, atol=1e-14)


def test_features_second_order_on_smooth_fields():
    errs = []
    for n in (16, 32, 64):
        L = 1000.0; h = L / n
        x = np.arange(n) * h
        xc = x + 0.5 * h
        k = 2 * np.pi / L
        zeta = np.arange(5) * 20.0
        nz = 4
        u = np.broadcast_to(np.sin(k * xc)[None, :, None], (nz, n, n)).copy()   # u(y) at x-faces
        th = 300.0 + np.broadcast_to(np.cos(k * xc)[None, None, :], (nz, n, n))
        st = _periodic_state(n, n, nz, fu=u, fth=th)
        f = M.features(*st, zeta, h, h, np.full(nz, 300.0))
        e1 = np.max(np.abs(f[..., 1] - k * np.cos(k * xc)[None, :, None]))       # du/dy
        e2 = np.max(np.abs(f[..., 9] + k * np.sin(k * xc)[None, None, :]))       # dtheta/dx
        errs.append(max(e1, e2))
    assert np.log2(errs[0] / errs[1]) > 1.9 and np.log2(errs[1] / errs[2]) > 1.9


def test_backscatter_clip_closed_form():
    """Pure strain S11 = 1, S22 = -1 with (Cs Delta)^2 = 1: Smagorinsky nu = 2, transfer 8, so the
    bound is -4.  A learned stress c S (transfer -2c) is scaled by 4/(2c) when 2c > 4 and left alone
    otherwise; forward scatter and the heat fluxes are never touched."""
    F = np.zeros((4, 12))
    F[:, 0], F[:, 4] = 1.0, -1.0
    c = np.array([10.0, 1.0, -10.0, 3.0])
    Y = np.zeros((4, 9))
    Y[:, 0], Y[:, 1] = c, -c
    Y[:, 6:] = [[0.1, 0.2, 0.3]] * 4
    out = M.clip_backscatter(Y, F, np.ones(4))
    S = M.strain_from_features(F)
    assert np.allclose(M.transfer(M.smagorinsky_stress(F, np.ones(4)), S), 8.0)
    np.testing.assert_allclose(out[0, :2], [2.0, -2.0])
    np.testing.assert_allclose(out[1:3], Y[1:3])
    np.testing.assert_allclose(out[3, :2], [4.0 / 6.0 * 3.0, -4.0 / 6.0 * 3.0])
    np.testing.assert_allclose(out[:, 6:], Y[:, 6:])


def test_backscatter_clip_bound_holds_for_random_stresses():
    rng = np.random.default_rng(5)
    F = rng.normal(size=(500, 12))
    d2 = rng.uniform(0.1, 2.0, size=500)
    Y = rng.normal(size=(500, 9)) * 3
    out = M.clip_backscatter(Y, F, d2)
    S = M.strain_from_features(F)
    lim = -0.5 * M.transfer(M.smagorinsky_stress(F, d2), S)
    t_in, t_out = M.transfer(Y[:, :6], S), M.transfer(out[:, :6], S)
    assert np.all(t_out >= lim - 1e-12 * np.abs(lim))
    keep = t_in >= lim
    np.testing.assert_array_equal(out[keep], Y[keep])
    assert np.any(~keep)
