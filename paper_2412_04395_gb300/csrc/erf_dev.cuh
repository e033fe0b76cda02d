// Device-side data structures and helpers of the GB300 dycore library.
//
// Geometry is kept separable: node heights are z(i,j,k) = zeta_k + s_k h(i,j) with
// s_k = (1 - zeta_k/z_t)^beta (Sec. 3.4 canonical form), so every metric of App. B at any
// point is a 1D vertical factor times a 2D terrain factor.  Only 1D (nz) and 2D (ny*nx) arrays
// are stored; the 3D metrics are formed in registers, which keeps them out of HBM traffic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace erfk {

constexpr double P00 = 1.0e5;          // EOS reference pressure (Sec. 2.1)
constexpr double RD = 287.0;           // dry-air gas constant
constexpr double CPD = 1004.5;         // specific heat at constant pressure
constexpr double CVD = CPD - RD;
constexpr double GAMMA = CPD / CVD;
constexpr double KAPPA = 0.4;          // von Karman constant (MOST)
constexpr double RV = 461.5;           // water-vapour gas constant (moist air, Sec. 2.1)
constexpr double LV = 2.5e6;           // latent heat of vaporisation (Kessler microphysics, Sec. 2.4)
constexpr double RHOW = 1000.0;        // liquid-water density (surface precipitation depth)

struct Geo {
    int nx, ny, nz;
    long long nxy, nc, nw;             // nx*ny, nx*ny*nz, nx*ny*(nz+1)
    double dx, dy, rdx, rdy;
    int terrain;
    // vertical 1D arrays
    const double *dzeta;   // [nz]   zeta_{k+1} - zeta_k
    const double *zetac;   // [nz]   (zeta_k + zeta_{k+1})/2
    const double *s;       // [nz+1] terrain decay factor at w-levels
    const double *sc;      // [nz]   (s_k + s_{k+1})/2
    const double *ds;      // [nz]   s_{k+1} - s_k
    const double *dzc;     // [nz+1] zetac_k - zetac_{k-1} (k = 1..nz-1)
    const double *delta2;  // [nz]   (Cs * (dx dy dzeta)^(1/3))^2 for Smagorinsky
    const double *rdzeta;  // [nz]   1 / dzeta
    const double *rdzc;    // [nz+1] 1 / dzc (k = 1..nz-1)
    const double *delta;   // [nz]   (dx dy dzeta)^(1/3), the filter width of the Deardorff closure
    // horizontal 2D terrain arrays [ny][nx]
    const double *hc;      // 4-node average of h (cell centre / w-face centre)
    const double *hxf;     // 2-node average of h along y (x-face)
    const double *hyf;     // 2-node average of h along x (y-face)
    const double *gxh;     // half the slope (hc_i - hc_{i-1})/dx at x-faces
    const double *gyh;     // half the slope (hc_j - hc_{j-1})/dy at y-faces
    const double *g4xq;    // a quarter of the 4th-order d hc/dx at cell centres
    const double *g4yq;
    // hydrostatic base state: [nz][ny][nx] with terrain, [nz] when flat
    const double *rho0, *th0, *p0;
    const double *qv0;     // base-state water vapour (moist handles; same layout as rho0), else null
    // reciprocal 3D metrics, terrain only ([nz][ny][nx]; null on flat grids): 1/H at cells,
    // x-faces and y-faces, 1/(z_c(k) - z_c(k-1)) at w-faces (k >= 1), and 1/(z_c(ku) - z_c(kl))
    // of the centred vertical difference at cells (kl = max(k-1, 0), ku = min(k+1, nz-1)).
    // An FP64 division costs ~10 FP64-pipe instructions, so each is taken once at init.
    const double *rH3, *rHx3, *rHy3, *rdzw3, *rdz2;
    const double *Hx3, *Hy3;   // terrain only: the heights H at x- and y-faces themselves
};

struct Phys {
    double g, f_cor, u_g, v_g, Cs, Pr_t, nu, z0, Qs, beta_s, beta_d, rPr_t;
    double b1, b2;        // substep off-centring weights (1 - beta_s)/2, (1 + beta_s)/2, formed on the host
    int closure, surface, scal_adv;
    int mom3;   // 1: upwind-3 momentum interpolant instead of upwind-5
    // Rayleigh damping (Sec. 3.7, App. D): rate ray_tau sin^2(pi/2 (z - ray_zd)/(ray_zt - ray_zd))
    // above ray_zd; ray_fields bitmask 1 u, 2 v, 4 w, 8 theta (0 = off)
    double ray_tau, ray_zd, ray_zt;
    int ray_fields;
    // moisture (Sec. 2.1, App. C): rho q_v, rho q_c, rho q_r of the stage state (null when dry)
    const double *rqv, *rqc, *rqr;
    int moist;
    // lateral relaxation zones (open x boundaries): rate relax_tau sin^2(pi/2 (1 - d/relax_w))
    // within relax_w of an x-edge of the domain of length Lx (relax_tau = 0: off)
    double relax_tau, relax_w, Lx;
    int anelastic;    // 1: anelastic equation set (Sec. 2.2): buoyancy rho0 g (theta - theta0) / theta0
};

// mixing ratios of the stage state at a cell: q_v + q_c (the 1/(1 + q_v + q_c) of Eq. mom) and
// (rho_m - rho_d) / rho_d = q_v + q_c + q_r; 0 on dry handles
__device__ __forceinline__ double q_vc(const Phys &ph, long long c, double rho) {
    return ph.moist ? (__ldg(ph.rqv + c) + __ldg(ph.rqc + c)) / rho : 0.0;
}
__device__ __forceinline__ double q_t(const Phys &ph, long long c, double rho) {
    return ph.moist ? (__ldg(ph.rqv + c) + __ldg(ph.rqc + c) + __ldg(ph.rqr + c)) / rho : 0.0;
}
__device__ __forceinline__ double relax_rate(const Phys &ph, double x) {
    const double d = fmin(x, ph.Lx - x);
    if (!(ph.relax_tau > 0.0) || !(d < ph.relax_w)) return 0.0;
    const double s = sin(0.5 * 3.141592653589793 * (1.0 - d / ph.relax_w));
    return ph.relax_tau * (s * s);
}

// Rayleigh damping rate at physical height z (0 below the damping layer)
__device__ __forceinline__ double ray_rate(const Phys &ph, double z) {
    if (!(z > ph.ray_zd)) return 0.0;
    const double s = sin(0.5 * 3.141592653589793 * (z - ph.ray_zd) / (ph.ray_zt - ph.ray_zd));
    return ph.ray_tau * (s * s);
}

// FP64 prognostic fields (cell, cell, x-face, y-face, w-face)
struct F5 {
    double *r, *t, *u, *v, *w;
};
struct CF5 {
    const double *r, *t, *u, *v, *w;
};

// face velocities, mass fluxes and rho*Omega of the stage state
struct Prep {
    const double *ux, *vy, *wz, *mfx, *mfy, *rom;
};
// stage LU factors of the vertical acoustic system at w-faces (rows k = 1..nz-1)
struct Tri {
    double *a, *cp, *im, *P, *Q;
};

// periodic wrap without integer division: one conditional correction covers the stencil
// offsets used here (|offset| <= 3) once n >= 4; smaller extents loop
__device__ __forceinline__ int wrapi(int i, int n) {
    if (n >= 4) {
        i += i < 0 ? n : 0;
        i -= i >= n ? n : 0;
        return i;
    }
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}
// even reflection of a cell level about the walls (ghost layers below/above the domain);
// one reflection covers k in [-3, nz+2] once nz >= 3
__device__ __forceinline__ int kref(int k, int nz) {
    if (nz >= 3) {
        k = k < 0 ? -1 - k : k;
        k = k >= nz ? 2 * nz - 1 - k : k;
        return k;
    }
    while (k < 0 || k >= nz) {
        if (k < 0) k = -1 - k;
        if (k >= nz) k = 2 * nz - 1 - k;
    }
    return k;
}
// linear indices in 32-bit arithmetic (grids are limited to fewer than 2^31 w-face points)
__device__ __forceinline__ long long cix(const Geo &g, int i, int j, int k) {
    return (long long)((k * g.ny + j) * g.nx + i);
}
__device__ __forceinline__ long long cixw(const Geo &g, int i, int j, int k) {
    return (long long)((k * g.ny + wrapi(j, g.ny)) * g.nx + wrapi(i, g.nx));
}
// cell value, periodic in x/y, reflected in z
__device__ __forceinline__ double cval(const Geo &g, const double *f, int i, int j, int k) {
    return __ldg(f + cixw(g, i, j, kref(k, g.nz)));
}
// w-face value, periodic in x/y, odd reflection about the wall values in z
__device__ __forceinline__ double wval(const Geo &g, const double *f, int i, int j, int k) {
    double sgn = 1.0, add = 0.0;
    while (k < 0 || k > g.nz) {
        if (k < 0) { add += sgn * 2.0 * __ldg(f + cixw(g, i, j, 0)); sgn = -sgn; k = -k; }
        else { add += sgn * 2.0 * __ldg(f + cixw(g, i, j, g.nz)); sgn = -sgn; k = 2 * g.nz - k; }
    }
    return add + sgn * __ldg(f + cixw(g, i, j, k));
}

// 1/x in FP64 by the Newton-Raphson iteration for the reciprocal, r <- r + r (1 - x r), from the
// hardware's approximate FP64 reciprocal (rcp.approx.ftz.f64); two steps take any estimate good
// to 2^-20 or better to rounding level.  Four FMAs on the FP64 pipe against about ten for a
// division, with no FP32 round trip.  Zero, subnormal, huge and non-finite x (an integer test of
// the exponent field) take the division.
__device__ __forceinline__ double rcp_d(double x) {
    const int e = (__double2hiint(x) >> 20) & 0x7ff;
    if (e < 64 || e > 1983) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// 1/x to about 2^-40 relative: the hardware's approximate FP64 reciprocal and one Newton step.
// For a quotient that only corrects a larger term (the WENO5 weighting, added to the middle
// candidate), where that error stays far below the rounding of the sum.  x must be a normal
// FP64 number.
__device__ __forceinline__ double rcp1_d(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return fma(r, fma(-x, r, 1.0), r);
}

// ---- metrics (App. B) in separable form
__device__ __forceinline__ int ij2(const Geo &g, int i, int j) { return wrapi(j, g.ny) * g.nx + wrapi(i, g.nx); }
__device__ __forceinline__ double Hc(const Geo &g, int i, int j, int k) {
    return g.terrain ? g.dzeta[k] + g.ds[k] * g.hc[ij2(g, i, j)] : g.dzeta[k];
}
// face heights: 1D on flat grids, tabulated over terrain (a load instead of an FP64 FMA)
__device__ __forceinline__ double Hx(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.Hx3 + cixw(g, i, j, k)) : g.dzeta[k];
}
__device__ __forceinline__ double Hy(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.Hy3 + cixw(g, i, j, k)) : g.dzeta[k];
}
// reciprocal heights: 1D tables on flat grids, 3D tables over terrain
__device__ __forceinline__ double rHc(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.rH3 + cixw(g, i, j, k)) : g.rdzeta[k];
}
__device__ __forceinline__ double rHxf(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.rHx3 + cixw(g, i, j, k)) : g.rdzeta[k];
}
__device__ __forceinline__ double rHyf(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.rHy3 + cixw(g, i, j, k)) : g.rdzeta[k];
}
__device__ __forceinline__ double rdzcw(const Geo &g, int i, int j, int k) {
    return g.terrain ? __ldg(g.rdzw3 + cixw(g, i, j, k)) : g.rdzc[k];
}
// terrain only: 1 / (z_c(ku) - z_c(kl)) of the centred vertical difference at cell (i,j,k)
__device__ __forceinline__ double rdz2c(const Geo &g, int i, int j, int k) {
    return __ldg(g.rdz2 + cixw(g, i, j, k));
}
__device__ __forceinline__ double zc(const Geo &g, int i, int j, int k) {
    return g.terrain ? g.zetac[k] + g.sc[k] * g.hc[ij2(g, i, j)] : g.zetac[k];
}
// h_xi / 2 and h_eta / 2 at x- and y-faces (the 1/2 of the two-point average they multiply); the
// w-face slopes carry the 1/4 of the four-point averages of the metric shift
__device__ __forceinline__ double hxi_x2(const Geo &g, int i, int j, int k) { return g.sc[k] * g.gxh[ij2(g, i, j)]; }
__device__ __forceinline__ double heta_y2(const Geo &g, int i, int j, int k) { return g.sc[k] * g.gyh[ij2(g, i, j)]; }
// the metric shift h_xi <U> + h_eta <V> at w-face (i,j,k) from the four-point sums au, av of U and V
__device__ __forceinline__ double w4_shift(const Geo &g, int i, int j, int k, double au, double av) {
    const int n = ij2(g, i, j);
    return g.s[k] * fma(g.g4xq[n], au, g.g4yq[n] * av);
}
__device__ __forceinline__ long long bix(const Geo &g, int i, int j, int k) {
    return g.terrain ? cixw(g, i, j, k) : (long long)k;
}

}  // namespace erfk
