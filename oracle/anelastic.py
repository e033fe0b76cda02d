"""FP64 oracle of the anelastic equation set (Sec. 2.2) with its time integration (Sec. 3.2).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg may use
it; the product path never does.  It shares no code with the CUDA library.

The slow tendencies come from the C oracle in its anelastic mode (rho held at the base density
rho0, the pressure perturbation p' taken from the projection instead of the EOS, buoyancy
rho0 g (theta - theta0) / theta0).  This module adds, in plain numpy:
  * SSP-RK2 (Shu & Osher 1988, as printed in Sec. 3.2):
        S*      = S^n + dt f(S^n),
        S^{n+1} = S^n + dt/2 (f(S^n) + f(S*)),
    each stage followed by the projection;
  * the projection of Sec. 3.2: solve dt div(grad psi) = div(rho0 u**) for psi, then
    rho0 u = rho0 u** - dt grad psi.  Readings where the paper is silent: the pressure after the
    first stage is p'* = p'^n + psi; after the second, whose provisional momentum carries the mean
    of the two stages' pressure gradients, p'^{n+1} = (p'^n + p'*)/2 + psi; the same dt scales
    both projections; the initial momentum is projected once before the first step;
  * the discrete operators of the C-grid: divergence at cells from face momenta (periodic x, y;
    no flux through the walls), gradient at faces from cell values; the Poisson operator is
    their composition, solved exactly by an FFT in x and y (the library FFT is one step here)
    and one tridiagonal system per horizontal wavenumber in z.  The (0, 0) mode, defined up to a
    constant, takes psi = 0 at the lowest level.
Flat grids only; nx and ny may be any size here.
"""
from __future__ import annotations

import numpy as np

MOM = ("rhou", "rhov", "rhow")


def divergence(mx, my, mz, dx, dy, dz):
    """Cell divergence of face fields: mx [nz][ny][nx] at x-faces (face i = left of cell i),
    my at y-faces, mz [nz+1][ny][nx] at w-faces; dz the nz cell heights."""
    return ((np.roll(mx, -1, axis=2) - mx) / dx + (np.roll(my, -1, axis=1) - my) / dy
            + (mz[1:] - mz[:-1]) / dz[:, None, None])


def gradient(psi, dx, dy, dzc):
    """Face gradients of a cell field: x-faces, y-faces, w-faces (interior only; 0 on the walls).
    dzc[k] = distance between the centres of cells k-1 and k (k = 1..nz-1)."""
    gx = (psi - np.roll(psi, 1, axis=2)) / dx
    gy = (psi - np.roll(psi, 1, axis=1)) / dy
    gz = np.zeros((psi.shape[0] + 1,) + psi.shape[1:])
    gz[1:-1] = (psi[1:] - psi[:-1]) / dzc[1:-1, None, None]
    return gx, gy, gz


def solve_poisson(rhs, dx, dy, dz, dzc):
    """psi with divergence(gradient(psi)) = rhs (rhs summing to zero per level weight dz)."""
    nz, ny, nx = rhs.shape
    R = np.fft.fft2(rhs, axes=(1, 2))
    lamx = -4.0 / dx ** 2 * np.sin(np.pi * np.arange(nx) / nx) ** 2
    lamy = -4.0 / dy ** 2 * np.sin(np.pi * np.arange(ny) / ny) ** 2
    a = lamy[:, None] + lamx[None, :]
    lo = np.zeros(nz)
    up = np.zeros(nz)
    for k in range(nz):
        if k >= 1:
            lo[k] = 1.0 / (dz[k] * dzc[k])
        if k <= nz - 2:
            up[k] = 1.0 / (dz[k] * dzc[k + 1])
    # Thomas algorithm over every wavenumber at once
    d = np.empty((nz, ny, nx))
    for k in range(nz):
        d[k] = a - lo[k] - up[k]
    rr = R.copy()
    uu = np.broadcast_to(up[:, None, None], (nz, ny, nx)).astype(complex).copy()
    # the (0, 0) mode: psi_0 = 0 replaces row 0
    d[0, 0, 0] = 1.0
    uu[0, 0, 0] = 0.0
    rr[0, 0, 0] = 0.0
    cp = np.empty((nz, ny, nx), dtype=complex)
    dp = np.empty((nz, ny, nx), dtype=complex)
    cp[0] = uu[0] / d[0]
    dp[0] = rr[0] / d[0]
    for k in range(1, nz):
        m = d[k] - lo[k] * cp[k - 1]
        cp[k] = uu[k] / m
        dp[k] = (rr[k] - lo[k] * dp[k - 1]) / m
    x = np.empty((nz, ny, nx), dtype=complex)
    x[-1] = dp[-1]
    for k in range(nz - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return np.fft.ifft2(x, axes=(1, 2)).real


class Anelastic:
    """SSP-RK2 steps of the anelastic equations on an oracle configured with anelastic = 1."""

    def __init__(self, o, project_initial=True):
        self.o = o
        c = o.cfg
        self.dx, self.dy, self.dt = c.dx, c.dy, c.dt
        H = o.geom("Hc")[:, 0, 0]
        zc = o.geom("zc")[:, 0, 0]
        self.dz = H
        self.dzc = np.zeros(c.nz + 1)
        self.dzc[1:-1] = zc[1:] - zc[:-1]
        if project_initial:
            m, _ = self.project({k: o.get(k) for k in MOM}, 1.0)
            for k in MOM:
                o.set(k, m[k])

    def project(self, M, dt):
        """The momentum with its divergence removed, and psi (dt div grad psi = div M)."""
        div = divergence(M["rhou"], M["rhov"], M["rhow"], self.dx, self.dy, self.dz)
        psi = solve_poisson(div / dt, self.dx, self.dy, self.dz, self.dzc)
        gx, gy, gz = gradient(psi, self.dx, self.dy, self.dzc)
        return {"rhou": M["rhou"] - dt * gx, "rhov": M["rhov"] - dt * gy, "rhow": M["rhow"] - dt * gz}, psi

    def div(self):
        o = self.o
        return divergence(o.get("rhou"), o.get("rhov"), o.get("rhow"), self.dx, self.dy, self.dz)

    def step(self, n=1):
        o, dt = self.o, self.dt
        keys = ("rhotheta",) + MOM
        rkey = {"rhotheta": "R_rhotheta", "rhou": "R_rhou", "rhov": "R_rhov", "rhow": "R_rhow"}
        for _ in range(n):
            Sn = {k: o.get(k) for k in keys}
            pn = o.get("p_anelastic")
            R1 = o.slow_rhs()
            S1 = {k: Sn[k] + dt * R1[rkey[k]] for k in keys}
            m, psi = self.project({k: S1[k] for k in MOM}, dt)
            S1.update(m)
            p1 = pn + psi
            for k in keys:
                o.set(k, S1[k])
            o.set("p_anelastic", p1)
            R2 = o.slow_rhs()
            S2 = {k: Sn[k] + 0.5 * dt * (R1[rkey[k]] + R2[rkey[k]]) for k in keys}
            m, psi = self.project({k: S2[k] for k in MOM}, dt)
            S2.update(m)
            for k in keys:
                o.set(k, S2[k])
            o.set("p_anelastic", 0.5 * (pn + p1) + psi)
