"""Seeded synthetic workloads: grids, terrain, initial perturbations and run parameters.

This module is shared by the CUDA path, the oracle, the tests and the benchmark.  It holds
none of the dycore's arithmetic: only the inputs (flat-column face heights, nodal terrain,
potential-temperature perturbations, face velocities) and the run parameters of each case.
The base state, the metrics and the conversion of a perturbation into conserved variables
are computed by each implementation on its own.

Cases (sizes and initial conditions of the paper's benchmark problems, Sec. 4 and Table D):
  density_current   2D-slab cold bubble, 256 x 4 x 64 at 100 m, Smagorinsky Cs = 0.17
  hill_bubble       3D warm bubble over a Gaussian hill, 256 x 256 x 128 at 50 m, stretched dz
  neutral_abl       neutral ABL LES, 1024 x 1024 x 128 at 10 m, MOST, Coriolis, seeded noise
  convective_abl    convective ABL, 2048 x 2048 x 160 at 40 m, surface heat flux 0.2 K m/s
Each builder takes smaller sizes for tests; spacing and physics stay those of the case.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# configuration enums shared by both implementations' wrappers (pure names, no arithmetic)
MOM_UPWIND3, MOM_UPWIND5 = 3, 5
SCAL_WENO5_JS, SCAL_WENO5_Z, SCAL_UPWIND3 = 0, 1, 3
CLOSURE_NONE, CLOSURE_CONST_NU, CLOSURE_SMAGORINSKY, CLOSURE_LEARNED, CLOSURE_DEARDORFF = 0, 1, 2, 3, 4
RAY_U, RAY_V, RAY_W, RAY_THETA = 1, 2, 4, 8
SURFACE_SLIP, SURFACE_MOST = 0, 1
PREC_FP64, PREC_MIXED32 = 0, 1


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    zeta: np.ndarray                       # nz+1 flat-column face heights [m], zeta[0] = 0
    terrain: Optional[np.ndarray] = None   # (ny, nx) nodal terrain heights [m] at (i dx, j dy)
    terrain_beta: int = 1
    dt: float = 0.25
    n_substeps: int = 6
    beta_s: float = 0.1
    beta_d: float = 0.1
    mom_adv: int = MOM_UPWIND5
    scal_adv: int = SCAL_WENO5_JS
    closure: int = CLOSURE_NONE
    Cs: float = 0.17
    Pr_t: float = 1.0 / 3.0
    nu: float = 0.0
    gravity: float = 9.81
    f_cor: float = 0.0
    u_g: float = 0.0
    v_g: float = 0.0
    surface: int = SURFACE_SLIP
    z0: float = 0.1
    sfc_theta_flux: float = 0.0
    theta_s: float = 300.0
    brunt_N: float = 0.0
    p_s: float = 1.0e5
    knots: Optional[tuple] = None          # (z[], theta[]) piecewise-linear sounding
    precision: int = PREC_FP64
    steps: int = 1
    # initial perturbation (potential temperature at cells) and face velocities
    dtheta: Optional[np.ndarray] = None
    u: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None
    w: Optional[np.ndarray] = None
    tracer: int = 0                        # 1: passive scalar rho phi (advanced after the substeps)
    phi: Optional[np.ndarray] = None       # initial phi at cells (tracer = 1)
    tke: Optional[np.ndarray] = None       # initial SGS kinetic energy e [m^2/s^2] at cells (closure 4)
    ray_tau: float = 0.0                   # Rayleigh damping strength at the top [1/s] (0 = off)
    ray_zd: float = 0.0                    # bottom of the damping layer [m]
    ray_fields: int = 0                    # RAY_U | RAY_V | RAY_W | RAY_THETA
    moist: int = 0                         # 1: rho q_v, rho q_c, rho q_r with Kessler microphysics
    qv_knots: Optional[tuple] = None       # (z[], q_v[]) base-state water-vapour sounding [kg/kg]
    qv: Optional[np.ndarray] = None        # initial q_v at cells (None: the base state's)
    qc: Optional[np.ndarray] = None        # initial cloud water / rain mixing ratios at cells
    qr: Optional[np.ndarray] = None
    relax_tau: float = 0.0                 # lateral relaxation zones (open x boundaries) [1/s]
    relax_width: float = 0.0               # their width [m]
    anelastic: int = 0                     # 1: the anelastic equation set (SSP-RK2 + projection)
    notes: str = ""

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def uniform_zeta(nz: int, dz: float) -> np.ndarray:
    return np.arange(nz + 1, dtype=np.float64) * dz


def stretched_zeta(nz: int, dz0: float, ratio: float) -> np.ndarray:
    """Face heights with dz_k = dz0 * ratio**k (bottom spacing + growth ratio, Sec. 3.4)."""
    dz = dz0 * ratio ** np.arange(nz, dtype=np.float64)
    return np.concatenate([[0.0], np.cumsum(dz)])


def cell_coords(nx, ny, zeta, dx, dy):
    """Cell-centre x, y and flat-column height zeta_c as [k][j][i] arrays."""
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    zc = 0.5 * (zeta[:-1] + zeta[1:])
    Z, Y, X = np.meshgrid(zc, y, x, indexing="ij")
    return X, Y, Z


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Counter-based generator (Steele, Lea & Flood 2014), uint64 arithmetic with wraparound."""
    z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def seeded_noise_at(index: np.ndarray, seed: int, amplitude: float) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude] from splitmix64(seed xor global cell index), at the
    given global cell indices (k ny + j) nx + i."""
    bits = splitmix64(np.asarray(index, dtype=np.uint64) ^ np.uint64(seed))
    u01 = (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amplitude * (2.0 * u01 - 1.0)


def seeded_noise(shape, seed: int, amplitude: float) -> np.ndarray:
    """seeded_noise_at over a whole [k][j][i] grid."""
    idx = np.arange(int(np.prod(shape)), dtype=np.uint64)
    return seeded_noise_at(idx, seed, amplitude).reshape(shape)


# ---------------------------------------------------------------------------------- cases
def density_current(nx=256, ny=4, nz=64, steps=100, dx=100.0, dt=0.25) -> Workload:
    """Straka cold bubble (Sec. 4.1.1): dT = -15 (cos(pi L) + 1)/2 for L < 1, radii 4 km / 2 km,
    centre z = 3 km; placed at the centre of a periodic domain (whole bubble, not the half
    domain with a symmetry plane).  Neutral theta0 = 300 K, Smagorinsky Cs = 0.17."""
    zeta = uniform_zeta(nz, dx)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    xc = 0.5 * nx * dx
    L = np.sqrt(((X - xc) / 4000.0) ** 2 + ((Z - 3000.0) / 2000.0) ** 2)
    dth = np.where(L < 1.0, -15.0 * 0.5 * (np.cos(np.pi * L) + 1.0), 0.0)
    return Workload("density_current", nx, ny, nz, dx, dx, zeta, dt=dt, n_substeps=6,
                    closure=CLOSURE_SMAGORINSKY, Cs=0.17, steps=steps, dtheta=dth,
                    notes="2D-slab cold-bubble density current, FP64, Smagorinsky")


def straka_density_current(nx=512, ny=4, nz=64, dx=100.0, dt=1.0, steps=900) -> Workload:
    """The literature form of the density current (Sec. 4.1.1): the -15 K cos^2 decrement is on
    temperature, so theta' = dT / pi0(z) with the Exner function of the neutral hydrostatic base
    state, pi0 = 1 - g z / (c_p theta0); constant nu = alpha_theta = 75 m^2/s, no turbulence model;
    dt 1 s at 100 m.  The periodic domain of 51.2 km with the bubble at its centre is the paper's
    half domain with the symmetry plane, mirrored (the fronts stay clear of the periodic images
    for 900 s)."""
    zeta = uniform_zeta(nz, dx)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    xc = 0.5 * nx * dx
    L = np.sqrt(((X - xc) / 4000.0) ** 2 + ((Z - 3000.0) / 2000.0) ** 2)
    dT = np.where(L < 1.0, -15.0 * 0.5 * (np.cos(np.pi * L) + 1.0), 0.0)
    pi0 = 1.0 - 9.81 * Z / (1004.5 * 300.0)
    return Workload("straka_density_current", nx, ny, nz, dx, dx, zeta, dt=dt, n_substeps=6,
                    closure=CLOSURE_CONST_NU, nu=75.0, Pr_t=1.0, steps=steps, dtheta=dT / pi0,
                    notes="Straka (1993) density current, constant nu = alpha = 75 m^2/s, FP64")


def dry_bubble(nx=200, ny=4, nz=100, dx=100.0, dt=0.5, steps=2000) -> Workload:
    """Dry rising bubble (Sec. 4.1.2, after Bryan & Fritsch 2002): theta0 = 300 K, surface
    pressure 1e5 Pa, +2 cos^2(pi r / 2) K for r < 1 with radius 2 km centred at z = 2 km in a
    20 km x 10 km domain (here periodic in x, the bubble at the centre), inviscid, dx = dz = 100 m,
    dt 0.5 s, 1000 s."""
    zeta = uniform_zeta(nz, dx)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    r = np.sqrt(((X - 0.5 * nx * dx) / 2000.0) ** 2 + ((Z - 2000.0) / 2000.0) ** 2)
    dth = np.where(r < 1.0, 2.0 * np.cos(0.5 * np.pi * r) ** 2, 0.0)
    return Workload("dry_bubble", nx, ny, nz, dx, dx, zeta, dt=dt, n_substeps=6, closure=CLOSURE_NONE,
                    steps=steps, dtheta=dth, notes="dry rising bubble, inviscid, FP64")


def gaussian_hill(nx, ny, dx, dy, h0=400.0, a=1000.0):
    """Nodal terrain h = h0 exp(-r^2/a^2) centred in the domain; nodes at (i dx, j dy)."""
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    Y, X = np.meshgrid(y, x, indexing="ij")
    xc, yc = 0.5 * nx * dx, 0.5 * ny * dy
    return h0 * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / a ** 2)


def hill_bubble(nx=256, ny=256, nz=128, steps=500, dx=50.0, dz0=20.0, ratio=1.015,
                h0=400.0, terrain=True) -> Workload:
    """Warm bubble (2 cos^2(pi r/2), Sec. 4.1.2 form) of +2 K, radius 500 m, centred 1 km above
    the domain centre (computational height), over a Gaussian hill h0 = 400 m, a = 1 km;
    theta0 = 300 exp(N^2 z/g), N = 0.01 1/s; stretched dz from 20 m; inviscid."""
    zeta = stretched_zeta(nz, dz0, ratio)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    xc, yc = 0.5 * nx * dx, 0.5 * ny * dx
    r = np.sqrt((X - xc) ** 2 + (Y - yc) ** 2 + (Z - 1000.0) ** 2) / 500.0
    dth = np.where(r < 1.0, 2.0 * np.cos(0.5 * np.pi * r) ** 2, 0.0)
    ter = gaussian_hill(nx, ny, dx, dx, h0=h0) if terrain else None
    return Workload("hill_bubble", nx, ny, nz, dx, dx, zeta, terrain=ter, terrain_beta=1,
                    dt=0.25, n_substeps=6, closure=CLOSURE_NONE, brunt_N=0.01, steps=steps,
                    dtheta=dth, notes="3D warm bubble over a Gaussian hill, FP64, inviscid")


def squall_line(nx=1500, ny=4, nz=240, dx=100.0, dt=0.25, steps=36000, relax_width=10000.0,
                relax_tau=0.01) -> Workload:
    """Idealised two-dimensional squall line (Sec. 4.1.3): 150 km x 24 km at 100 m, dt 0.25 s,
    constant diffusivities nu = alpha = 200 m^2/s for every variable, Kessler microphysics, open
    lateral boundaries (here relaxation zones of relax_width toward the initial state at rate
    relax_tau), slip walls at the ground and the lid.  Warm bubble dtheta = 3 cos^2(pi r / 2),
    r < 1, centre (75 km, 2 km), radii 10 km x 1.5 km; wind u = -12 + 0.0048 z below 2.5 km, 0 above.
    Sounding (the paper names a moist, subsaturated hydrostatic background without printing it):
    theta after Weisman & Klemp (1982), 300 K at the ground rising as (z/12 km)^(5/4) to 343 K at
    the 12 km tropopause and isothermal (213 K) above; water vapour by piecewise-linear knots from
    14 g/kg at the ground, decreasing with height (subsaturated everywhere)."""
    zeta = uniform_zeta(nz, dx)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    xc = 0.5 * nx * dx
    r = np.sqrt(((X - xc) / 10000.0) ** 2 + ((Z - 2000.0) / 1500.0) ** 2)
    dth = np.where(r < 1.0, 3.0 * np.cos(0.5 * np.pi * r) ** 2, 0.0)
    zf = Z  # u sits at x-faces, at the cell-centre height
    u = np.where(zf <= 2500.0, -12.0 + 0.0048 * zf, 0.0)
    top = max(nz * dx, 12001.0)
    zk = np.concatenate([np.linspace(0.0, 12000.0, 25), [top + 1.0]])
    thk = np.where(zk <= 12000.0, 300.0 + 43.0 * (np.minimum(zk, 12000.0) / 12000.0) ** 1.25,
                   343.0 * np.exp(9.81 * (zk - 12000.0) / (1004.5 * 213.0)))
    qz = np.array([0.0, 1000.0, 2000.0, 4000.0, 6000.0, 8000.0, 10000.0, 12000.0, top + 1.0])
    qk = np.array([14.0, 11.0, 8.0, 4.0, 1.6, 0.5, 0.12, 0.02, 0.01]) * 1.0e-3
    return Workload("squall_line", nx, ny, nz, dx, dx, zeta, dt=dt, n_substeps=6, closure=CLOSURE_CONST_NU,
                    nu=200.0, Pr_t=1.0, knots=(zk, thk), steps=steps, dtheta=dth, u=u, moist=1,
                    qv_knots=(qz, qk), relax_tau=relax_tau, relax_width=relax_width,
                    notes="2D squall line, Kessler microphysics, FP64")


NOISE_SEED = 20241205
NOISE_TOP = 400.0   # seeded theta noise below this height [m]


def _abl_common(nx, ny, nz, dx, knots, noise_top, steps, dt, name, flux, precision):
    zeta = uniform_zeta(nz, dx)
    X, Y, Z = cell_coords(nx, ny, zeta, dx, dx)
    noise = seeded_noise((nz, ny, nx), NOISE_SEED, 0.25)
    dth = np.where(Z < noise_top, noise, 0.0)
    u = np.full((nz, ny, nx), 10.0)
    return Workload(name, nx, ny, nz, dx, dx, zeta, dt=dt, n_substeps=10,
                    closure=CLOSURE_SMAGORINSKY, Cs=0.17, f_cor=1.0e-4, u_g=10.0, v_g=0.0,
                    surface=SURFACE_MOST, z0=0.1, sfc_theta_flux=flux, knots=knots,
                    precision=precision, steps=steps, dtheta=dth, u=u)


def neutral_abl(nx=1024, ny=1024, nz=128, steps=100, dx=10.0, precision=PREC_MIXED32) -> Workload:
    """Neutral ABL LES: theta 300 K to 500 m, +10 K/km to 650 m, +3 K/km above; U = U_g = 10 m/s;
    MOST z0 = 0.1 m; f = 1e-4 1/s; seeded uniform theta noise of +-0.25 K below 400 m."""
    top = nz * dx
    knots = (np.array([0.0, 500.0, 650.0, max(top, 651.0)]),
             np.array([300.0, 300.0, 301.5, 301.5 + 3.0e-3 * (max(top, 651.0) - 650.0)]))
    return _abl_common(nx, ny, nz, dx, knots, NOISE_TOP, steps, 0.1, "neutral_abl", 0.0, precision)


def convective_abl(nx=2048, ny=2048, nz=160, steps=1000, dx=40.0, precision=PREC_MIXED32) -> Workload:
    """Convective ABL: theta 300 K mixed to 1 km, +5 K over 100 m, then +3 K/km; surface
    kinematic heat flux 0.2 K m/s; U_g = 10 m/s; noise as the neutral case."""
    top = nz * dx
    knots = (np.array([0.0, 1000.0, 1100.0, max(top, 1101.0)]),
             np.array([300.0, 300.0, 305.0, 305.0 + 3.0e-3 * (max(top, 1101.0) - 1100.0)]))
    return _abl_common(nx, ny, nz, dx, knots, NOISE_TOP, steps, 0.4, "convective_abl", 0.2, precision)


def paper_scaling(nx=512, ny=512, nz=256, steps=100, dx=4.0, precision=PREC_FP64) -> Workload:
    """The paper's scaling workload (Sec. 5.2): a neutral ABL LES on 512 x 512 x 256 cells over
    2048 x 2048 x 1024 m (4 m spacing) with third-order upwind advection of momenta and scalars
    and Smagorinsky.  Sounding, wind, roughness, Coriolis and noise are the neutral case's; the
    time step is the neutral case's scaled to the 4 m spacing (0.04 s, 10 substeps)."""
    top = nz * dx
    knots = (np.array([0.0, 500.0, 650.0, max(top, 651.0)]),
             np.array([300.0, 300.0, 301.5, 301.5 + 3.0e-3 * (max(top, 651.0) - 650.0)]))
    wl = _abl_common(nx, ny, nz, dx, knots, NOISE_TOP, steps, 0.04, "paper_scaling", 0.0, precision)
    return wl.with_(mom_adv=MOM_UPWIND3, scal_adv=SCAL_UPWIND3)


def abl_window(case, nx_full: int, ny_full: int, i0: int, j0: int, nx: int, ny: int, **kw) -> Workload:
    """The nx x ny columns starting at (i0, j0) (periodic wrap) of an ABL case (neutral_abl,
    convective_abl or paper_scaling) of nx_full x ny_full columns, as a periodic workload of its
    own: the same levels, sounding and settings, and the full case's initial noise at those
    columns (drawn at their global cell indices, so no full-size array is built)."""
    wl = case(nx=nx, ny=ny, **kw)
    ii = (i0 + np.arange(nx)) % nx_full
    jj = (j0 + np.arange(ny)) % ny_full
    K, J, I = np.meshgrid(np.arange(wl.nz, dtype=np.uint64), jj.astype(np.uint64), ii.astype(np.uint64),
                          indexing="ij")
    noise = seeded_noise_at((K * np.uint64(ny_full) + J) * np.uint64(nx_full) + I, NOISE_SEED, 0.25)
    zc = 0.5 * (wl.zeta[:-1] + wl.zeta[1:])
    dth = np.where(zc[:, None, None] < NOISE_TOP, noise, 0.0)
    return wl.with_(dtheta=dth, notes=wl.notes + f" (window {nx}x{ny} at ({i0}, {j0}) of {nx_full}x{ny_full})")


def smooth_velocity(nx_full: int, ny_full: int, nz: int, seed: int, amplitude: float, i0: int = 0, j0: int = 0,
                    nx: Optional[int] = None, ny: Optional[int] = None, modes: int = 6, kmax: int = 48):
    """Resolved velocity perturbations (u', v', w') of a periodic domain of nx_full x ny_full columns
    and nz levels, on the nx x ny columns from (i0, j0) (default: the whole domain): for each
    component a sum of `modes` separable Fourier modes sin(2 pi kx x + a) cos(2 pi ky y + b) with
    integer wavenumbers 1..kmax over the domain and seeded amplitudes and phases, times the vertical
    envelope sin(pi z / z_top).  u' sits at x-faces, v' at y-faces, w' at w-faces (zero at both
    walls).  Being a formula of the global position, any window of it equals the whole field
    restricted to those columns."""
    nx = nx_full if nx is None else nx
    ny = ny_full if ny is None else ny
    rng = np.random.default_rng(seed)
    ii = (i0 + np.arange(nx)) % nx_full
    jj = (j0 + np.arange(ny)) % ny_full
    out = []
    for comp in range(3):
        xs = (ii + (0.0 if comp == 0 else 0.5)) / nx_full        # u at x-faces, v and w at centres
        ys = (jj + (0.0 if comp == 1 else 0.5)) / ny_full
        zs = (np.arange(nz + 1) / nz) if comp == 2 else ((np.arange(nz) + 0.5) / nz)
        plane = np.zeros((ny, nx))
        for _ in range(modes):
            a = amplitude * rng.standard_normal() / np.sqrt(modes)
            kx, ky = rng.integers(1, kmax + 1, size=2)
            px, py = rng.uniform(0.0, 2.0 * np.pi, size=2)
            plane += a * np.outer(np.cos(2.0 * np.pi * ky * ys + py), np.sin(2.0 * np.pi * kx * xs + px))
        env = np.sin(np.pi * zs)
        if comp == 2:
            env[0] = env[-1] = 0.0
        out.append(env[:, None, None] * plane[None])
    return tuple(out)


def with_tracer(wl: Workload, kind: str = "blob", radius_frac: float = 0.2) -> Workload:
    """The same case with a passive scalar: phi = 1 everywhere ("one") or a Gaussian blob
    exp(-r^2/R^2), R = radius_frac x the domain width, centred in x and y at a third of the
    column height ("blob")."""
    if kind == "one":
        return wl.with_(tracer=1, phi=np.ones((wl.nz, wl.ny, wl.nx)))
    X, Y, Z = cell_coords(wl.nx, wl.ny, wl.zeta, wl.dx, wl.dy)
    R = radius_frac * wl.nx * wl.dx
    zc = wl.zeta[-1] / 3.0
    r2 = (X - 0.5 * wl.nx * wl.dx) ** 2 + (Y - 0.5 * wl.ny * wl.dy) ** 2 * (wl.ny > 4) + (Z - zc) ** 2
    return wl.with_(tracer=1, phi=np.exp(-r2 / R ** 2))


CASES = {
    "squall_line": squall_line,
    "density_current": density_current,
    "hill_bubble": hill_bubble,
    "neutral_abl": neutral_abl,
    "convective_abl": convective_abl,
    "paper_scaling": paper_scaling,
}
