"""FP64 oracle of the learned subgrid closure (numpy; test infrastructure only).

The paper names surrogate models as future work (Sec. 6) and fixes nothing about them; the
closure takes these readings:
  * features at cell centres of a flat C-grid: the 9 resolved velocity gradients du_i/dx_j,
    dtheta/dx, dtheta/dy and N^2 = g/theta0 dtheta/dz (12 inputs);
  * MLP 12 -> 64 -> 64 -> 64 -> 9, SiLU hidden activations, linear output;
  * outputs: kinematic SGS stress t_ij (11, 22, 33, 12, 13, 23) [m^2/s^2] and heat flux h_j [K m/s],
    standardised with training-set mean/std (inputs likewise);
  * targets from a Favre 4x4x4 box filter of a fine run:
        rho_bar = <rho>,  u~_i = <rho u_i>/rho_bar,  t_ij = <rho u_i u_j>/rho_bar - u~_i u~_j,
        h_j = <rho u_j theta>/rho_bar - u~_j theta~;
  * loss: mean squared error on standardised outputs; optimiser Adam (Kingma & Ba 2015);
  * at inference, backscatter is limited: where the learned stress transfers energy from the
    subgrid to the resolved scales at more than half the Smagorinsky dissipation rate
    (-t_ij S_ij < -0.5 Pi_s), the six stresses are scaled so that -t_ij S_ij = -0.5 Pi_s.
Everything here is written from those definitions, in plain numpy, independent of the CUDA code.
"""
from __future__ import annotations

import numpy as np

LAYERS = (12, 64, 64, 64, 9)
N_IN, N_OUT = 12, 9


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 has float32's exponent range and 8 significant bits: a finite value a = m 2^e
    (1/2 <= |m| < 1) is a multiple of the quantum q = 2^(max(e, -125) - 8), so normal numbers keep
    8 bits and everything below 2^-126 is a multiple of the subnormal quantum 2^-133.  The value
    is rounded once, straight from float64 (no intermediate float32 rounding), to the nearest
    multiple of its quantum with exact halves going to the even multiple; a result of magnitude
    2^128 or more is an infinity (the largest finite bfloat16 is 255 * 2^120).  Signed zeros,
    infinities and NaNs pass through."""
    a = np.asarray(x, dtype=np.float64)
    finite = np.isfinite(a)
    af = np.where(finite, a, 0.0)
    _, e = np.frexp(af)
    q = np.ldexp(1.0, np.maximum(e, -125) - 8)
    r = np.round(af / q) * q            # a / q is exact (a power-of-two scaling); round = half-even
    r = np.where(np.abs(r) >= 2.0 ** 128, np.copysign(np.inf, af), r)
    r = np.where(af == 0.0, af, r)      # keeps the sign of zero
    return np.where(finite, r, a)


def forward(params, X, bf16_inputs=False):
    """params: list of (W [out, in], b [out]); X [n, 12] standardised.  Returns (Y, cache).
    bf16_inputs: round every layer's input activations and weights to bfloat16 (as tensor-core
    inference does; products and sums stay in float64)."""
    a = np.asarray(X, dtype=np.float64)
    cache = [a]
    for l, (W, b) in enumerate(params):
        if bf16_inputs:
            z = bf16(a) @ bf16(W).T + b
        else:
            z = a @ W.T + b
        if l < len(params) - 1:
            cache.append(z)
            a = silu(z)
            cache.append(a)
        else:
            a = z
    return a, cache


def pack_blob(params, in_mean, in_std, out_mean, out_std, version=1):
    """Closure blob: uint32 magic 'ERFM', uint32 version, FP32 stats and parameters."""
    flat = [np.asarray(in_mean), np.asarray(in_std), np.asarray(out_mean), np.asarray(out_std)]
    for W, b in params:
        flat += [np.asarray(W).ravel(), np.asarray(b).ravel()]
    body = np.concatenate(flat).astype(np.float32)
    head = np.array([0x4D465245, version], dtype=np.uint32)
    return head.tobytes() + body.tobytes()


def unpack_params(vec):
    """Parameter list from the flat 9737-vector W1 b1 W2 b2 W3 b3 W4 b4."""
    out, o = [], 0
    for a, b in zip(LAYERS[:-1], LAYERS[1:]):
        W = np.asarray(vec[o:o + a * b], dtype=np.float64).reshape(b, a); o += a * b
        bb = np.asarray(vec[o:o + b], dtype=np.float64); o += b
        out.append((W, bb))
    return out


def flatten_params(params):
    return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in params])


def backward(params, cache, dY):
    """Gradients of a scalar loss with dL/dY = dY (reverse-mode chain rule through the layers)."""
    grads = [None] * len(params)
    g = np.asarray(dY, dtype=np.float64)
    L = len(params)
    for l in range(L - 1, -1, -1):
        W, b = params[l]
        a_in = cache[0] if l == 0 else cache[2 * l]
        grads[l] = (g.T @ a_in, g.sum(axis=0))
        if l > 0:
            z_prev = cache[2 * l - 1]
            g = (g @ W) * dsilu(z_prev)
    return grads


def mse(Y, T):
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_init(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params], \
           [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t >= 1): biased moments, bias correction, parameter step."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p, gp, mp, vp in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mp = b1 * mp + (1.0 - b1) * gp
            vp = b2 * vp + (1.0 - b2) * gp * gp
            mh = mp / (1.0 - b1 ** t)
            vh = vp / (1.0 - b2 ** t)
            new.append((p - lr * mh / (np.sqrt(vh) + eps), mp, vp))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def train(params, X, T, epochs, batch, lr=1e-3):
    """Mini-batch Adam over the samples in the given order (last partial batch included)."""
    m, v = adam_init(params)
    t = 0
    n = len(X)
    losses = []
    for ep in range(epochs):
        for s in range(0, n, batch):
            xb, tb = X[s:s + batch], T[s:s + batch]
            Y, cache = forward(params, xb)
            loss, dY = mse(Y, tb)
            grads = backward(params, cache, dY)
            t += 1
            params, m, v = adam_step(params, grads, m, v, t, lr)
            losses.append(loss)
    return params, losses


# ------------------------------------------------------------------ features and filter
def _centre_vel(ru, rv, rw, rho):
    """Cell-centre velocities of a periodic flat C-grid state [k][j][i]."""
    rx = 0.5 * (np.roll(rho, 1, axis=2) + rho)
    ry = 0.5 * (np.roll(rho, 1, axis=1) + rho)
    ux = ru / rx
    vy = rv / ry
    nz = rho.shape[0]
    rz = np.empty_like(rw)
    rz[1:nz] = 0.5 * (rho[:-1] + rho[1:])
    rz[0] = rho[0]
    rz[nz] = rho[-1]
    wz = rw / rz
    uc = 0.5 * (ux + np.roll(ux, -1, axis=2))
    vc = 0.5 * (vy + np.roll(vy, -1, axis=1))
    wc = 0.5 * (wz[:-1] + wz[1:])
    return ux, vy, wz, uc, vc, wc


def _ddz_c(f, zc):
    """d/dz of a cell field: centred over cell centres, one-sided at the walls."""
    d = np.empty_like(f)
    nz = f.shape[0]
    if nz == 1:
        return np.zeros_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (zc[2:] - zc[:-2])[:, None, None]
    d[0] = (f[1] - f[0]) / (zc[1] - zc[0])
    d[-1] = (f[-1] - f[-2]) / (zc[-1] - zc[-2])
    return d


def features(rho, rt, ru, rv, rw, zeta, dx, dy, theta0, g=9.81):
    """The 12 closure inputs at every cell of a flat periodic C-grid state ([k][j][i] arrays;
    theta0 = base potential temperature per level).  Diagonal gradients from face differences,
    cross gradients from centred differences of cell-centre velocities."""
    ux, vy, wz, uc, vc, wc = _centre_vel(ru, rv, rw, rho)
    dz = np.diff(zeta)
    zc = 0.5 * (zeta[:-1] + zeta[1:])
    th = rt / rho
    cx = lambda f: (np.roll(f, -1, axis=2) - np.roll(f, 1, axis=2)) / (2 * dx)
    cy = lambda f: (np.roll(f, -1, axis=1) - np.roll(f, 1, axis=1)) / (2 * dy)
    f = np.empty(rho.shape + (12,))
    f[..., 0] = (np.roll(ux, -1, axis=2) - ux) / dx          # du/dx
    f[..., 1] = cy(uc)                                      # du/dy
    f[..., 2] = _ddz_c(uc, zc)                              # du/dz
    f[..., 3] = cx(vc)                                      # dv/dx
    f[..., 4] = (np.roll(vy, -1, axis=1) - vy) / dy          # dv/dy
    f[..., 5] = _ddz_c(vc, zc)                              # dv/dz
    f[..., 6] = cx(wc)                                      # dw/dx
    f[..., 7] = cy(wc)                                      # dw/dy
    f[..., 8] = (wz[1:] - wz[:-1]) / dz[:, None, None]      # dw/dz
    f[..., 9] = cx(th)                                      # dtheta/dx
    f[..., 10] = cy(th)                                     # dtheta/dy
    f[..., 11] = g / theta0[:, None, None] * _ddz_c(th, zc)  # N^2
    return f


def box_filter(rho, rt, ru, rv, rw, r=4):
    """Favre r x r x r box filter of a fine flat state: coarse C-grid state (cell means of rho,
    rho theta; face means of the face momenta) and SGS targets t_ij, h_j at coarse cells."""
    nz, ny, nx = rho.shape
    Nz, Ny, Nx = nz // r, ny // r, nx // r
    ux, vy, wz, uc, vc, wc = _centre_vel(ru, rv, rw, rho)
    th = rt / rho

    def cmean(f):
        return f.reshape(Nz, r, Ny, r, Nx, r).mean(axis=(1, 3, 5))

    rb = cmean(rho)
    Rt = cmean(rt)
    # coarse x-face I = fine x-face r*I; average over its r x r fine faces in (j, k)
    Ru = ru[:, :, ::r].reshape(Nz, r, Ny, r, Nx).mean(axis=(1, 3))
    Rv = rv[:, ::r, :].reshape(Nz, r, Ny, Nx, r).mean(axis=(1, 4))
    Rw = rw[::r].reshape(Nz + 1, Ny, r, Nx, r).mean(axis=(2, 4))
    vel = (uc, vc, wc)
    ut = [cmean(rho * q) / rb for q in vel]
    tht = Rt / rb
    T = np.empty((Nz, Ny, Nx, 9))
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for n, (a, b) in enumerate(pairs):
        T[..., n] = cmean(rho * vel[a] * vel[b]) / rb - ut[a] * ut[b]
    for j in range(3):
        T[..., 6 + j] = cmean(rho * vel[j] * th) / rb - ut[j] * tht
    return (rb, Rt, Ru, Rv, Rw), T


def strain_from_features(F):
    """Resolved strain-rate components (S11, S22, S33, S12, S13, S23) from the 12 features."""
    F = np.asarray(F, dtype=np.float64)
    return np.stack([F[..., 0], F[..., 4], F[..., 8], 0.5 * (F[..., 1] + F[..., 3]),
                     0.5 * (F[..., 2] + F[..., 6]), 0.5 * (F[..., 5] + F[..., 7])], axis=-1)


def smagorinsky_stress(F, delta2):
    """Kinematic Smagorinsky-Lilly stress -2 nu (S_ij - S_kk delta_ij / 3), nu = delta2 sqrt(2 S:S),
    delta2 = (Cs Delta)^2 per cell; order 11, 22, 33, 12, 13, 23."""
    S = strain_from_features(F)
    SS = S[..., 0] ** 2 + S[..., 1] ** 2 + S[..., 2] ** 2 + 2 * (S[..., 3] ** 2 + S[..., 4] ** 2 + S[..., 5] ** 2)
    nu = np.asarray(delta2) * np.sqrt(2 * SS)
    tr = (S[..., 0] + S[..., 1] + S[..., 2]) / 3
    dev = S.copy()
    dev[..., :3] -= tr[..., None]
    return -2 * nu[..., None] * dev


def transfer(tau, S):
    """Resolved-to-subgrid energy transfer -t_ij S_ij of a symmetric stress (6 components)."""
    return -(tau[..., 0] * S[..., 0] + tau[..., 1] * S[..., 1] + tau[..., 2] * S[..., 2]
             + 2 * (tau[..., 3] * S[..., 3] + tau[..., 4] * S[..., 4] + tau[..., 5] * S[..., 5]))


def clip_backscatter(Y, F, delta2):
    """Y [n, 9] kinematic learned outputs, F [n, 12] features, delta2 [n]: the six stresses of each
    cell whose transfer is below -0.5 x the Smagorinsky transfer are scaled onto that bound."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    S = strain_from_features(F)
    pl = transfer(Y[:, :6], S)
    ps = transfer(smagorinsky_stress(F, delta2), S)
    lim = -0.5 * ps
    bad = pl < lim
    Y[bad, :6] *= (lim[bad] / pl[bad])[:, None]
    return Y


def standardise_stats(A):
    """Per-column mean and standard deviation (a zero deviation is replaced by 1)."""
    mu = A.reshape(-1, A.shape[-1]).mean(axis=0)
    sd = A.reshape(-1, A.shape[-1]).std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return mu, sd


# ------------------------------------------------------------------ the closure inside a step
def unpack_blob(blob: bytes):
    """Inverse of pack_blob: (params, in_mean, in_std, out_mean, out_std), the FP32 values as
    float64."""
    head = np.frombuffer(blob[:8], dtype=np.uint32)
    assert head[0] == 0x4D465245, "not a closure blob"
    body = np.frombuffer(blob[8:], dtype=np.float32).astype(np.float64)
    st, vec = body[:2 * N_IN + 2 * N_OUT], body[2 * N_IN + 2 * N_OUT:]
    in_mu, in_sd = st[:N_IN], st[N_IN:2 * N_IN]
    out_mu, out_sd = st[2 * N_IN:2 * N_IN + N_OUT], st[2 * N_IN + N_OUT:]
    return unpack_params(vec), in_mu, in_sd, out_mu, out_sd


class LearnedClosure:
    """The learned SGS model of a stage state on a flat periodic C-grid, as the step uses it:
    features -> standardise -> network (BF16 operands, as the tensor cores take them) ->
    de-standardise -> backscatter limit; Smagorinsky-Lilly in any cell whose standardised input
    leaves |z| <= 6 or whose output is not finite.  Returns the nine density-weighted
    cell-centre planes rho t11, t22, t33, t12, t13, t23, rho h1, h2, h3.

    Each call records the fallback count and the smallest distance of a cell's max |z| from the
    threshold 6 (self.margin), so a test can tell whether a decision was close enough to the
    threshold for FP32 and FP64 inputs to take it differently."""

    def __init__(self, blob, zeta, dx, dy, theta0, Cs, Pr_t, g=9.81, bf16_operands=True):
        self.params, self.in_mu, self.in_sd, self.out_mu, self.out_sd = unpack_blob(blob)
        self.zeta, self.dx, self.dy = np.asarray(zeta, dtype=np.float64), dx, dy
        self.theta0 = np.asarray(theta0, dtype=np.float64)
        self.Pr_t, self.g, self.bf16 = Pr_t, g, bf16_operands
        dz = np.diff(self.zeta)
        self.delta2 = (Cs * np.cbrt(dx * dy * dz)) ** 2       # (Cs Delta)^2 per level
        self.margin = np.inf
        self.fallbacks = []

    def __call__(self, rho, rt, ru, rv, rw):
        F = features(rho, rt, ru, rv, rw, self.zeta, self.dx, self.dy, self.theta0, self.g)
        shp = rho.shape
        Fn = F.reshape(-1, N_IN)
        d2 = np.broadcast_to(self.delta2[:, None, None], shp).reshape(-1)
        Z = (Fn - self.in_mu) / self.in_sd
        zmax = np.max(np.abs(Z), axis=1)
        self.margin = min(self.margin, float(np.min(np.abs(zmax - 6.0))))
        fb = ~(zmax <= 6.0)
        Y, _ = forward(self.params, Z, bf16_inputs=self.bf16)
        Y = Y * self.out_sd + self.out_mu
        fb |= ~np.all(np.isfinite(Y), axis=1)
        Y = clip_backscatter(np.where(np.isfinite(Y), Y, 0.0), Fn, d2)
        # Smagorinsky-Lilly fallback: stress -2 nu dev(S), heat flux -nu/Pr_t grad(theta)
        S = strain_from_features(Fn)
        SS = S[:, 0] ** 2 + S[:, 1] ** 2 + S[:, 2] ** 2 + 2 * (S[:, 3] ** 2 + S[:, 4] ** 2 + S[:, 5] ** 2)
        nu = d2 * np.sqrt(2 * SS)
        zc = 0.5 * (self.zeta[:-1] + self.zeta[1:])
        dthdz = _ddz_c(rt / rho, zc).reshape(-1)
        Ys = np.empty_like(Y)
        Ys[:, :6] = smagorinsky_stress(Fn, d2)
        Ys[:, 6] = -nu / self.Pr_t * Fn[:, 9]
        Ys[:, 7] = -nu / self.Pr_t * Fn[:, 10]
        Ys[:, 8] = -nu / self.Pr_t * dthdz
        out = np.where(fb[:, None], Ys, Y) * rho.reshape(-1)[:, None]
        self.fallbacks.append(int(np.sum(fb)))
        return out.T.reshape((N_OUT,) + shp)
