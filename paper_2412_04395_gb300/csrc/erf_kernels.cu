// FP64 kernels of one RK3 step of the compressible dycore (arXiv 2412.04395, Sec. 3.1 + App. C).
//
// One thread per output point; neighbours come through the read-only cache.  Periodic x/y by
// index wrap, walls by reflected ghost levels.  The kernel sequence of one stage is
//   stage_begin (EOS: p', pi, theta; perturbations X'' = S^n - S^t; Omega'')
//   prep        (face velocities, mass fluxes, rho*Omega)
//   flux_theta + rhs_cells, flux_u + rhs_u, flux_v + rhs_v, flux_w + rhs_w   (slow tendencies
//               R^t: each advective face flux once, then its divergence with the pressure
//               gradient, buoyancy and Coriolis)
//   sgs_edges, sgs_mu, sgs_tau, sgs_div   (subgrid terms, with a closure or MOST)
//   tri_build   (per column: coefficients of the vertical acoustic system and their LU
//               factors, fixed for the stage)
//   n_s x { sub_horiz, sub_expl, sub_col, sub_fin }   (App. C substeps)
//   stage_end   (S^t <- S^t + X'')
#include "erf_dev.cuh"
#include "erf_launch.h"
#include "erf_stencil.cuh"

#include <math.h>

namespace erfk {

// the upwind side of an advecting momentum m: the left one for m >= 0, by an integer test of the
// sign bit (an FP64 comparison would take the FP64 pipe, the bound of these kernels).  -0 takes
// the right side; every caller multiplies the interpolated value by that zero.
__device__ __forceinline__ bool upwind_left(double m) { return __double2hiint(m) >= 0; }

// Exner function and pressure from rho*theta (Sec. 2.1 EOS, dry):
// pi = (R_d rho theta / P00)^(R_d/c_v), p = R_d rho theta pi.  The product is rounded on its
// own (__dmul_rn) so that a later p - p0 cannot be contracted into an FMA: the base state is
// subtracted exactly and an undisturbed column keeps p' = 0 bit for bit.
__device__ __forceinline__ void eos_pi(double rt, double &p, double &pi) {
    // pi = x^(R_d/c_v) with x = R_d rho theta / P00 and R_d/c_v = 2/5, so pi = x z with
    // z = a^(-1/5), a = x^3.  z starts from an FP32 estimate z0 (relative error ~1e-7) and takes
    // one step of the binomial series of the correction: with r = 1 - a z0^5, z = z0 (1 - r)^(-1/5)
    // = z0 (1 + r/5 + 3 r^2/25 + O(r^3)), so the error becomes O(r^3) ~ 1e-21, below rounding (no
    // division; 8 FP64 multiply/FMA for the root instead of a general pow).
    static_assert(RD / CVD == 0.4, "this form of the EOS assumes R_d/c_v = 2/5");
    double x = RD * rt * (1.0 / P00);
    double a = x * x * x;
    double z = (double)exp2f(-0.6f * log2f((float)x));
    double z2 = z * z;
    double r = fma(-a, z2 * z2 * z, 1.0);
    z = fma(z, fma(0.12, r, 0.2) * r, z);
    pi = x * z;
    p = __dmul_rn(RD * rt, pi);
}

// ------------------------------------------------------------------ init: terrain + base state
__global__ void k_terrain_avg(Geo g, const double *hn, double *hc, double *hxf, double *hyf) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.nxy) return;
    int i = n % g.nx, j = n / g.nx;
    double h00 = hn[ij2(g, i, j)], h10 = hn[ij2(g, i + 1, j)], h01 = hn[ij2(g, i, j + 1)], h11 = hn[ij2(g, i + 1, j + 1)];
    hc[n] = 0.25 * (h00 + h10 + h01 + h11);
    hxf[n] = 0.5 * (h00 + h01);
    hyf[n] = 0.5 * (h00 + h10);
}

__global__ void k_terrain_grad(Geo g, const double *hc, double *gxh, double *gyh, double *g4xq, double *g4yq) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.nxy) return;
    int i = n % g.nx, j = n / g.nx;
    // stored as half the slope (and the 4th-order slope as a quarter): the pressure-gradient
    // correction multiplies h_xi by the 1/2 of a two-point average, the metric shift by the 1/4 of
    // a four-point average; both scalings are exact
    gxh[n] = 0.5 * ((hc[n] - hc[ij2(g, i - 1, j)]) * g.rdx);
    gyh[n] = 0.5 * ((hc[n] - hc[ij2(g, i, j - 1)]) * g.rdy);
    g4xq[n] = 0.25 * ((hc[ij2(g, i - 2, j)] - hc[ij2(g, i + 2, j)] + 8.0 * (hc[ij2(g, i + 1, j)] - hc[ij2(g, i - 1, j)])) / (12.0 * g.dx));
    g4yq[n] = 0.25 * ((hc[ij2(g, i, j - 2)] - hc[ij2(g, i, j + 2)] + 8.0 * (hc[ij2(g, i, j + 1)] - hc[ij2(g, i, j - 1)])) / (12.0 * g.dy));
}

// reciprocal 3D metrics over terrain (built once; the step kernels multiply by them)
__global__ void k_terrain_recip(Geo g, double *Hx3, double *Hy3, double *rH3, double *rHx3, double *rHy3,
                                double *rdzw3, double *rdz2) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double hc = g.hc[ij2(g, i, j)];
    rH3[c] = 1.0 / (g.dzeta[k] + g.ds[k] * hc);
    const double hx = g.dzeta[k] + g.ds[k] * g.hxf[ij2(g, i, j)], hy = g.dzeta[k] + g.ds[k] * g.hyf[ij2(g, i, j)];
    Hx3[c] = hx;
    Hy3[c] = hy;
    rHx3[c] = 1.0 / hx;
    rHy3[c] = 1.0 / hy;
    rdzw3[c] = k >= 1 ? 1.0 / (g.dzc[k] + (g.sc[k] - g.sc[k - 1]) * hc) : 0.0;
    int kl = k == 0 ? 0 : k - 1, ku = k == g.nz - 1 ? g.nz - 1 : k + 1;
    rdz2[c] = ku > kl ? 1.0 / ((g.zetac[ku] + g.sc[ku] * hc) - (g.zetac[kl] + g.sc[kl] * hc)) : 0.0;
}

struct ThetaProfile {
    int n_knots;
    const double *kz, *kt;   // device copies
    double theta_s, N, g;
};
__device__ double theta0_of(const ThetaProfile &tp, double z) {
    if (tp.n_knots > 0) {
        if (z <= tp.kz[0]) return tp.kt[0];
        for (int n = 1; n < tp.n_knots; ++n)
            if (z <= tp.kz[n]) {
                double t = (z - tp.kz[n - 1]) / (tp.kz[n] - tp.kz[n - 1]);
                return tp.kt[n - 1] + t * (tp.kt[n] - tp.kt[n - 1]);
            }
        return tp.kt[tp.n_knots - 1];
    }
    if (tp.N == 0.0 || tp.g == 0.0) return tp.theta_s;
    return tp.theta_s * exp(tp.N * tp.N * z / tp.g);
}
// rho from p and theta (EOS inverted): rho = (P00 / (R_d theta)) (p/P00)^(1/gamma)
__device__ __forceinline__ double rho_from(double p, double th) {
    return (P00 / (RD * th)) * pow(p * (1.0 / P00), 1.0 / GAMMA);
}

// Hydrostatic base state per column (Sec. 3.8): trapezoidal dp/dz = -rho g between cell
// centres, starting from p_s at z = 0, each level solved by Newton-Raphson for p; then
// p0 is re-evaluated by the EOS of rho0 theta0 so the undisturbed state has p' = 0.
// base-state water vapour q_v0(z): piecewise-linear sounding, constant beyond its ends
struct QvProfile {
    int n;
    const double *kz, *kq;
};
__device__ double qv0_of(const QvProfile &qp, double z) {
    if (qp.n <= 0) return 0.0;
    if (z <= qp.kz[0]) return qp.kq[0];
    for (int m = 1; m < qp.n; ++m)
        if (z <= qp.kz[m]) {
            double t = (z - qp.kz[m - 1]) / (qp.kz[m] - qp.kz[m - 1]);
            return qp.kq[m - 1] + t * (qp.kq[m] - qp.kq[m - 1]);
        }
    return qp.kq[qp.n - 1];
}
// total density rho_d (1 + q_v) from p, theta_d and q_v by the moist EOS of Sec. 2.1
__device__ __forceinline__ double rho_m_from(double p, double th, double q) {
    return rho_from(p, th * (1.0 + (RV / RD) * q)) * (1.0 + q);
}

__global__ void k_base_state(Geo g, ThetaProfile tp, QvProfile qp, double p_s, double grav, double *rho0,
                             double *th0, double *p0, double *qv0) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long ncol = g.terrain ? g.nxy : 1;
    if (n >= ncol) return;
    int i = (int)(n % g.nx), j = (int)(n / g.nx);
    const bool moist = qv0 != nullptr;
    double p_prev = p_s, z_prev = 0.0;
    double r_prev = moist ? rho_m_from(p_s, theta0_of(tp, 0.0), qv0_of(qp, 0.0)) : rho_from(p_s, theta0_of(tp, 0.0));
    for (int k = 0; k < g.nz; ++k) {
        double z = zc(g, i, j, k), th = theta0_of(tp, z), dz = z - z_prev;
        double q = moist ? qv0_of(qp, z) : 0.0;
        double p = p_prev - grav * dz * r_prev;
        for (int it = 0; it < 50; ++it) {
            double r = moist ? rho_m_from(p, th, q) : rho_from(p, th);
            double f = p - p_prev + 0.5 * grav * dz * (r_prev + r);
            double df = 1.0 + 0.5 * grav * dz * r / (GAMMA * p);
            double dp = -f / df;
            p += dp;
            if (fabs(dp) <= 1.0e-14 * fabs(p)) break;
        }
        double r = moist ? rho_m_from(p, th, q) : rho_from(p, th);
        long long b = g.terrain ? cix(g, i, j, k) : k;
        rho0[b] = r;          // total density on moist handles
        th0[b] = th;
        double pp, pie;
        if (moist) {
            qv0[b] = q;
            eos_pi(r / (1.0 + q) * th * (1.0 + (RV / RD) * q), pp, pie);
        } else {
            eos_pi(r * th, pp, pie);
        }
        p0[b] = pp;
        p_prev = p; r_prev = r; z_prev = z;
    }
}

// initial state from a theta perturbation at unchanged pressure
__global__ void k_init_cells(Geo g, const double *dth, double *rho, double *rt) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    long long b = bix(g, i, j, k);
    double th = g.th0[b] + (dth ? dth[c] : 0.0);
    double t = g.rho0[b] * g.th0[b];
    rt[c] = t;
    rho[c] = g.rho0[b] * (g.th0[b] / th);   // rho0 theta0 / theta, exactly rho0 when dtheta = 0
}
// moist handles: water vapour q_v at cells (null: the base state's q_v0), pressure unchanged,
// rho_d theta_d (1 + (R_v/R_d) q_v) = rho_d0 theta0 (1 + (R_v/R_d) q_v0), rho_d0 = rho0 / (1 + q_v0);
// no cloud or rain
__global__ void k_init_cells_moist(Geo g, const double *dth, const double *qv, double *rho, double *rt,
                                   double *rqv, double *rqc, double *rqr) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    long long b = bix(g, i, j, k);
    double th = g.th0[b] + (dth ? dth[c] : 0.0);
    double q0 = g.qv0[b], q = qv ? qv[c] : q0;
    double rd0 = g.rho0[b] / (1.0 + q0), f = (1.0 + (RV / RD) * q0) / (1.0 + (RV / RD) * q);
    rt[c] = rd0 * g.th0[b] * f;
    double r = rd0 * (g.th0[b] / th) * f;
    rho[c] = r;
    rqv[c] = r * q;
    rqc[c] = 0.0;
    rqr[c] = 0.0;
}
__global__ void k_init_faces(Geo g, const double *u, const double *v, const double *w, const double *rho,
                             double *ru, double *rv, double *rw) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    if (k < g.nz) {
        ru[n] = u ? u[n] * 0.5 * (cval(g, rho, i - 1, j, k) + rho[n]) : 0.0;
        rv[n] = v ? v[n] * 0.5 * (cval(g, rho, i, j - 1, k) + rho[n]) : 0.0;
    }
    rw[n] = w ? w[n] * 0.5 * (cval(g, rho, i, j, k - 1) + cval(g, rho, i, j, k)) : 0.0;
}

// h_xi <U> + h_eta <V> at w-face (i,j,k) with the 4-point averages of App. B (levels outside
// the domain reflected)
__device__ __forceinline__ double metric_shift(const Geo &g, const double *U, const double *V, int i, int j, int k) {
    // four-point sums; the 1/4 of the averages is in the slope tables, the level factor s_k is
    // applied once to both terms
    double au = cval(g, U, i, j, k - 1) + cval(g, U, i + 1, j, k - 1) + cval(g, U, i, j, k) + cval(g, U, i + 1, j, k);
    double av = cval(g, V, i, j, k - 1) + cval(g, V, i, j + 1, k - 1) + cval(g, V, i, j, k) + cval(g, V, i, j + 1, k);
    return w4_shift(g, i, j, k, au, av);
}

// walls: Omega = 0 at k = 0 (rho w = metric shift of the horizontal momenta) and rho w = 0 at the top
__global__ void k_wall_bc(Geo g, const double *ru, const double *rv, double *rw) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nxy) return;
    int i = (int)(n % g.nx), j = (int)(n / g.nx);
    rw[n] = g.terrain ? metric_shift(g, ru, rv, i, j, 0) : 0.0;
    rw[cix(g, i, j, g.nz)] = 0.0;
}

// ------------------------------------------------------------------ stage begin
// EOS at the stage state; X'' = S^n - S^t; Theta''_prev = Theta''; Omega'' = W'' - metric shift
__global__ void k_stage_begin(Geo g, CF5 sn, CF5 st, F5 x, double *pp, double *pi, double *th,
                              double *Tprev, double *Om, const double *rqv) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    if (k < g.nz) {
        double rt = st.t[n], rho = st.r[n];
        double p, pie;
        // the moist EOS (Sec. 2.1) with the stage's q_v, else the dry one
        if (rqv) eos_pi(rt * (1.0 + (RV / RD) * (rqv[n] / rho)), p, pie);
        else eos_pi(rt, p, pie);
        long long b = bix(g, i, j, k);
        pp[n] = p - g.p0[b];
        pi[n] = pie;
        th[n] = rt * rcp_d(rho);
        x.r[n] = sn.r[n] - rho;
        double xt = sn.t[n] - rt;
        x.t[n] = xt;
        Tprev[n] = xt;
        x.u[n] = sn.u[n] - st.u[n];
        x.v[n] = sn.v[n] - st.v[n];
    }
    double xw = sn.w[n] - st.w[n];
    x.w[n] = xw;
    if (k == 0 || k == g.nz) { Om[n] = 0.0; return; }
    double om = xw;
    if (g.terrain) {
        double au = 0.0, av = 0.0;
        for (int dk = -1; dk <= 0; ++dk) {
            for (int di = 0; di <= 1; ++di) {
                long long a = cixw(g, i + di, j, k + dk);
                au += sn.u[a] - st.u[a];
            }
            for (int dj = 0; dj <= 1; ++dj) {
                long long a = cixw(g, i, j + dj, k + dk);
                av += sn.v[a] - st.v[a];
            }
        }
        om -= w4_shift(g, i, j, k, au, av);
    }
    Om[n] = om;
}

// face velocities (momentum / face-averaged density), mass fluxes per unit length, rho*Omega
__global__ void k_prep(Geo g, CF5 st, double *ux, double *vy, double *wz, double *mfx, double *mfy, double *rom) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    if (k < g.nz) {
        double r = st.r[n];
        double ru = st.u[n], rv = st.v[n];
        ux[n] = ru * rcp_d(0.5 * (cval(g, st.r, i - 1, j, k) + r));
        vy[n] = rv * rcp_d(0.5 * (cval(g, st.r, i, j - 1, k) + r));
        mfx[n] = Hx(g, i, j, k) * ru;
        mfy[n] = Hy(g, i, j, k) * rv;
    }
    double rb = 0.5 * (cval(g, st.r, i, j, k - 1) + cval(g, st.r, i, j, k));
    double rw = st.w[n];
    wz[n] = rw * rcp_d(rb);
    if (k == 0 || k == g.nz) rom[n] = 0.0;
    else rom[n] = g.terrain ? rw - metric_shift(g, st.u, st.v, i, j, k) : rw;
}

// ------------------------------------------------------------------ SGS (Sec. 2.3, reading R6)
struct Vel {
    const double *ux, *vy, *wz;
};
// strain components at the three edge types, with slip walls (S13 = S23 = 0 on k = 0, nz)
__device__ __forceinline__ double S12e(const Geo &g, const Vel &v, int i, int j, int k) {
    return 0.5 * ((cval(g, v.ux, i, j, k) - cval(g, v.ux, i, j - 1, k)) * g.rdy
                + (cval(g, v.vy, i, j, k) - cval(g, v.vy, i - 1, j, k)) * g.rdx);
}
__device__ __forceinline__ double S13e(const Geo &g, const Vel &v, int i, int j, int k) {
    if (k <= 0 || k >= g.nz) return 0.0;
    double rdz = g.rdzc[k];
    return 0.5 * ((cval(g, v.ux, i, j, k) - cval(g, v.ux, i, j, k - 1)) * rdz
                + (__ldg(v.wz + cixw(g, i, j, k)) - __ldg(v.wz + cixw(g, i - 1, j, k))) * g.rdx);
}
__device__ __forceinline__ double S23e(const Geo &g, const Vel &v, int i, int j, int k) {
    if (k <= 0 || k >= g.nz) return 0.0;
    double rdz = g.rdzc[k];
    return 0.5 * ((cval(g, v.vy, i, j, k) - cval(g, v.vy, i, j, k - 1)) * rdz
                + (__ldg(v.wz + cixw(g, i, j, k)) - __ldg(v.wz + cixw(g, i, j - 1, k))) * g.rdy);
}
__device__ __forceinline__ void diag_strain(const Geo &g, const Vel &v, int i, int j, int k, double &s11, double &s22, double &s33) {
    s11 = (cval(g, v.ux, i + 1, j, k) - cval(g, v.ux, i, j, k)) * g.rdx;
    s22 = (cval(g, v.vy, i, j + 1, k) - cval(g, v.vy, i, j, k)) * g.rdy;
    s33 = (__ldg(v.wz + cixw(g, i, j, k + 1)) - __ldg(v.wz + cixw(g, i, j, k))) * g.rdzeta[k];
}

// mu = rho (Cs Delta)^2 sqrt(2 S_ij S_ij) (Smagorinsky-Lilly) or rho nu (constant); the
// off-diagonal strains come from the edge arrays of k_sgs_edges (4-point averages to the centre)
// eddy viscosity at cells and the deviatoric diagonal stresses -2 mu (S_ii - div/3) (t11, t22, t33)
// Deardorff (closure 4, Sec. 2.3; Deardorff 1980 with the coefficients of Moeng 1984): from the
// SGS energy e = max(rho e / rho, 0) and N^2 = (g/theta) dtheta/dz (centred, one-sided at the
// walls), l = Delta or 0.76 sqrt(e)/N when shorter in stable air, K_m = 0.1 l sqrt(e),
// K_h = (1 + 2 l/Delta) K_m; mu = rho K_m, muh = rho K_h and the local part of the energy source
// rho (P + B - eps) with P = 2 K_m (S_ij S_ij - (S_kk)^2/3) (what the stress -2 mu (S - D) takes
// from the resolved flow), B = -K_h N^2, eps = (0.19 + 0.51 l/Delta) e^(3/2)/l.  Flat grids.
struct Tke {
    const double *rtke, *th;
    double *muh, *src;
};
__global__ void k_sgs_mu(Geo g, Phys ph, Vel v, const double *rho, const double *e12, const double *e13,
                         const double *e23, double *mu, double *t11, double *t22, double *t33, Tke tk) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double m = 0.0;
    double s11, s22, s33;
    diag_strain(g, v, i, j, k, s11, s22, s33);
    if (ph.closure == 2 || ph.closure == 4) {
        double s12 = 0.25 * (cval(g, e12, i, j, k) + cval(g, e12, i + 1, j, k) + cval(g, e12, i, j + 1, k) + cval(g, e12, i + 1, j + 1, k));
        double s13 = 0.25 * (__ldg(e13 + cixw(g, i, j, k)) + __ldg(e13 + cixw(g, i + 1, j, k)) + __ldg(e13 + cixw(g, i, j, k + 1))
                           + __ldg(e13 + cixw(g, i + 1, j, k + 1)));
        double s23 = 0.25 * (__ldg(e23 + cixw(g, i, j, k)) + __ldg(e23 + cixw(g, i, j + 1, k)) + __ldg(e23 + cixw(g, i, j, k + 1))
                           + __ldg(e23 + cixw(g, i, j + 1, k + 1)));
        double SS = s11 * s11 + s22 * s22 + s33 * s33 + 2.0 * (s12 * s12 + s13 * s13 + s23 * s23);
        if (ph.closure == 2) {
            m = rho[c] * g.delta2[k] * sqrt(2.0 * SS);
        } else {
            const double r = rho[c];
            const double e = fmax(__ldg(tk.rtke + c) / r, 0.0);
            const double se = sqrt(e);
            const double D = g.delta[k];
            const int kl = k == 0 ? 0 : k - 1, ku = k == g.nz - 1 ? g.nz - 1 : k + 1;
            double N2 = 0.0;
            if (ku > kl)
                N2 = ph.g / __ldg(tk.th + c) * (cval(g, tk.th, i, j, ku) - cval(g, tk.th, i, j, kl))
                   / (g.zetac[ku] - g.zetac[kl]);
            double l = D;
            if (N2 > 0.0 && e > 0.0) l = fmin(D, 0.76 * se / sqrt(N2));
            const double Km = 0.1 * l * se;
            const double Kh = (1.0 + 2.0 * l / D) * Km;
            const double dv3 = s11 + s22 + s33;
            m = r * Km;
            tk.muh[c] = r * Kh;
            const double P = 2.0 * Km * (SS - dv3 * dv3 / 3.0);
            const double eps = (0.19 + 0.51 * l / D) * e * se / l;
            tk.src[c] = r * (P - Kh * N2 - eps);
        }
    } else if (ph.closure == 1) {
        m = rho[c] * ph.nu;
    }
    mu[c] = m;
    const double dv = (s11 + s22 + s33) * (1.0 / 3.0);
    t11[c] = -2.0 * m * (s11 - dv);
    t22[c] = -2.0 * m * (s22 - dv);
    t33[c] = -2.0 * m * (s33 - dv);
}

// MOST friction velocity (reading R15): neutral start, 5 fixed-point iterations through the
// Obukhov length with Businger-Dyer psi_m, z1/L clipped to [-5, 1].
__device__ double ustar_most(double U, double z1, double z0, double Q, double theta, double grav) {
    double lz = log(z1 / z0);
    double us = KAPPA * U / lz;
    if (Q == 0.0 || grav == 0.0) return us;
    for (int it = 0; it < 5; ++it) {
        double zeta;
        if (us <= 0.0) zeta = (Q > 0.0) ? -5.0 : 1.0;
        else zeta = z1 / (-us * us * us * theta / (KAPPA * grav * Q));
        zeta = fmin(fmax(zeta, -5.0), 1.0);
        double psi;
        if (zeta < 0.0) {
            double x = pow(1.0 - 16.0 * zeta, 0.25);
            psi = 2.0 * log(0.5 * (1.0 + x)) + log(0.5 * (1.0 + x * x)) - 2.0 * atan(x) + 0.5 * M_PI;
        } else {
            psi = -5.0 * zeta;
        }
        us = KAPPA * U / (lz - psi);
    }
    return us;
}

// MOST surface stresses (Sec. 3.8, reading R15) at the ground: tau13 at the x-face (i, j), tau23 at
// the y-face (i, j), -rho u*^2 u_i / |U| with the first-level wind; 0 for a slip wall
__device__ double most13(const Geo &g, const Phys &ph, const Vel &v, const double *rho, const double *th, int i, int j) {
    if (ph.surface != 1) return 0.0;
    double u = cval(g, v.ux, i, j, 0);
    double vv = 0.25 * (cval(g, v.vy, i - 1, j, 0) + cval(g, v.vy, i, j, 0) + cval(g, v.vy, i - 1, j + 1, 0) + cval(g, v.vy, i, j + 1, 0));
    double U = sqrt(u * u + vv * vv);
    if (!(U > 0.0)) return 0.0;
    double thf = 0.5 * (cval(g, th, i - 1, j, 0) + cval(g, th, i, j, 0));
    double rhf = 0.5 * (cval(g, rho, i - 1, j, 0) + cval(g, rho, i, j, 0));
    double z1 = 0.5 * g.dzeta[0];
    double us = ustar_most(U, z1, ph.z0, ph.Qs, thf, ph.g);
    return -rhf * us * us * u / U;
}
__device__ double most23(const Geo &g, const Phys &ph, const Vel &v, const double *rho, const double *th, int i, int j) {
    if (ph.surface != 1) return 0.0;
    double u = 0.25 * (cval(g, v.ux, i, j - 1, 0) + cval(g, v.ux, i + 1, j - 1, 0) + cval(g, v.ux, i, j, 0) + cval(g, v.ux, i + 1, j, 0));
    double vv = cval(g, v.vy, i, j, 0);
    double U = sqrt(u * u + vv * vv);
    if (!(U > 0.0)) return 0.0;
    double thf = 0.5 * (cval(g, th, i, j - 1, 0) + cval(g, th, i, j, 0));
    double rhf = 0.5 * (cval(g, rho, i, j - 1, 0) + cval(g, rho, i, j, 0));
    double z1 = 0.5 * g.dzeta[0];
    double us = ustar_most(U, z1, ph.z0, ph.Qs, thf, ph.g);
    return -rhf * us * us * vv / U;
}
// rho alpha dtheta/dn at the three face types (minus the diffusive flux); bottom face: the
// upward MOST flux rho Q enters as -rho Q
// The heat diffusivity rho alpha_theta is hs * hk at cells: mu / Pr_t (hk = mu, hs = 1/Pr_t), or
// rho K_h of the Deardorff closure (hk = muh, hs = 1).
__device__ __forceinline__ double heat_x(const Geo &g, double hs, const double *hk, const double *th, int i, int j, int k) {
    return 0.5 * (cval(g, hk, i - 1, j, k) + cval(g, hk, i, j, k)) * hs * (cval(g, th, i, j, k) - cval(g, th, i - 1, j, k)) * g.rdx;
}
__device__ __forceinline__ double heat_y(const Geo &g, double hs, const double *hk, const double *th, int i, int j, int k) {
    return 0.5 * (cval(g, hk, i, j - 1, k) + cval(g, hk, i, j, k)) * hs * (cval(g, th, i, j, k) - cval(g, th, i, j - 1, k)) * g.rdy;
}
__device__ __forceinline__ double heat_z(const Geo &g, const Phys &ph, double hs, const double *hk, const double *th,
                                         const double *rho, int i, int j, int k, int visc) {
    if (k == 0) return ph.surface == 1 ? -cval(g, rho, i, j, 0) * ph.Qs : 0.0;   // upward flux rho Q
    if (k >= g.nz || !visc) return 0.0;
    return 0.5 * (cval(g, hk, i, j, k - 1) + cval(g, hk, i, j, k)) * hs
         * (cval(g, th, i, j, k) - cval(g, th, i, j, k - 1)) * g.rdzc[k];
}

// The subgrid stress divergence, each strain and stress evaluated once: edge strains (k_sgs_edges),
// the eddy viscosity (k_sgs_mu), the edge stresses in place with MOST at the bottom (k_sgs_tau),
// then one kernel differences them into R_U, R_V, R_W and adds the heat-flux divergence to
// R_Theta.  Edge arrays: xy-edges [nz] levels, xz- and yz-edges [nz+1] w-levels.
#define SGS_CELL3D_W()                                              \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;            \
    if (i >= g.nx) return;                                          \
    const int j = blockIdx.y, k = blockIdx.z;                       \
    const long long n = ((long long)k * g.ny + j) * g.nx + i;
__global__ void k_sgs_edges(Geo g, Vel v, double *e12, double *e13, double *e23) {
    SGS_CELL3D_W();
    if (k < g.nz) e12[n] = S12e(g, v, i, j, k);
    e13[n] = S13e(g, v, i, j, k);
    e23[n] = S23e(g, v, i, j, k);
}
__global__ void k_sgs_tau(Geo g, Phys ph, Vel v, const double *mu, const double *rho, const double *th, int visc,
                          double *t12, double *t13, double *t23) {
    SGS_CELL3D_W();
    if (k < g.nz) {
        double me = 0.25 * (cval(g, mu, i - 1, j - 1, k) + cval(g, mu, i, j - 1, k) + cval(g, mu, i - 1, j, k) + cval(g, mu, i, j, k));
        t12[n] = visc ? -2.0 * me * t12[n] : 0.0;
    }
    if (k == 0) {
        t13[n] = most13(g, ph, v, rho, th, i, j);
        t23[n] = most23(g, ph, v, rho, th, i, j);
    } else if (k >= g.nz || !visc) {
        t13[n] = 0.0;
        t23[n] = 0.0;
    } else {
        double mx = 0.25 * (cval(g, mu, i - 1, j, k - 1) + cval(g, mu, i, j, k - 1) + cval(g, mu, i - 1, j, k) + cval(g, mu, i, j, k));
        double my = 0.25 * (cval(g, mu, i, j - 1, k - 1) + cval(g, mu, i, j, k - 1) + cval(g, mu, i, j - 1, k) + cval(g, mu, i, j, k));
        t13[n] = -2.0 * mx * t13[n];
        t23[n] = -2.0 * my * t23[n];
    }
}
__global__ void k_sgs_div(Geo g, Phys ph, const double *hk, double hs, const double *t11, const double *t22,
                          const double *t33, const double *rho, const double *th, int visc, const double *t12,
                          const double *t13, const double *t23, F5 R) {
    SGS_CELL3D_W();
    const long long nxy = g.nxy;
    if (k < g.nz) {
        double du = 0.0, dv = 0.0, hd = 0.0;
        if (visc) {
            du = (__ldg(t11 + n) - __ldg(t11 + cixw(g, i - 1, j, k))) * g.rdx
               + (__ldg(t12 + cixw(g, i, j + 1, k)) - __ldg(t12 + n)) * g.rdy;
            dv = (__ldg(t12 + cixw(g, i + 1, j, k)) - __ldg(t12 + n)) * g.rdx
               + (__ldg(t22 + n) - __ldg(t22 + cixw(g, i, j - 1, k))) * g.rdy;
            hd = (heat_x(g, hs, hk, th, i + 1, j, k) - heat_x(g, hs, hk, th, i, j, k)) * g.rdx
               + (heat_y(g, hs, hk, th, i, j + 1, k) - heat_y(g, hs, hk, th, i, j, k)) * g.rdy;
        }
        du += (__ldg(t13 + n + nxy) - __ldg(t13 + n)) * g.rdzeta[k];
        dv += (__ldg(t23 + n + nxy) - __ldg(t23 + n)) * g.rdzeta[k];
        hd += (heat_z(g, ph, hs, hk, th, rho, i, j, k + 1, visc) - heat_z(g, ph, hs, hk, th, rho, i, j, k, visc)) * rHc(g, i, j, k);
        R.u[n] -= du;
        R.v[n] -= dv;
        R.t[n] += hd;
    }
    if (visc && k >= 1 && k < g.nz) {
        double dw = (__ldg(t13 + cixw(g, i + 1, j, k)) - __ldg(t13 + n)) * g.rdx
                  + (__ldg(t23 + cixw(g, i, j + 1, k)) - __ldg(t23 + n)) * g.rdy
                  + (__ldg(t33 + n) - __ldg(t33 + n - nxy)) * rdzcw(g, i, j, k);
        R.w[n] -= dw;
    }
}

// transport of the SGS energy by the SGS eddies (Deardorff): div(2 mu grad e) added to the
// source, face coefficient the mean of the two cells' 2 mu (mu = rho K_m), e = max(rho e / rho, 0),
// no flux through the walls.  Flat grids.
__global__ void k_tke_diff(Geo g, const double *mu, const double *rtke, const double *rho, double *src) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    // e at a stencil point from the Newton reciprocal of rho (four FMAs; a division takes ~ten
    // FP64-pipe operations)
    auto ev = [&](int ii, int jj, int kk) {
        const long long q = cixw(g, ii, jj, kk);
        return fmax(__ldg(rtke + q) * rcp_d(__ldg(rho + q)), 0.0);
    };
    const double m0 = __ldg(mu + c), e0 = ev(i, j, k);
    const double fxm = (cval(g, mu, i - 1, j, k) + m0) * (e0 - ev(i - 1, j, k)) * g.rdx;
    const double fxp = (m0 + cval(g, mu, i + 1, j, k)) * (ev(i + 1, j, k) - e0) * g.rdx;
    const double fym = (cval(g, mu, i, j - 1, k) + m0) * (e0 - ev(i, j - 1, k)) * g.rdy;
    const double fyp = (m0 + cval(g, mu, i, j + 1, k)) * (ev(i, j + 1, k) - e0) * g.rdy;
    double fzm = 0.0, fzp = 0.0;
    if (k > 0) fzm = (__ldg(mu + c - g.nxy) + m0) * (e0 - ev(i, j, k - 1)) * g.rdzc[k];
    if (k < g.nz - 1) fzp = (m0 + __ldg(mu + c + g.nxy)) * (ev(i, j, k + 1) - e0) * g.rdzc[k + 1];
    src[c] += (fxp - fxm) * g.rdx + (fyp - fym) * g.rdy + (fzp - fzm) * g.rdzeta[k];
}

// moisture diffusion (Eqs. nonprecip, precip): src_q = div(rho alpha_q grad q) for q_v, q_c, q_r,
// rho alpha_q = hs * hk (the heat diffusivity of the closure), face coefficient the mean of the
// two cells, no flux through the walls.  Flat grids.
struct Q3 {
    const double *q[3];
};
struct Q3w {
    double *q[3];
};
__global__ void k_moist_diff(Geo g, const double *hk, double hs, Q3 rq, const double *rho, Q3w src) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    const double h0 = __ldg(hk + c);
    const double hxm = cval(g, hk, i - 1, j, k), hxp = cval(g, hk, i + 1, j, k);
    const double hym = cval(g, hk, i, j - 1, k), hyp = cval(g, hk, i, j + 1, k);
    // the seven stencil points and their reciprocal densities, shared by the three species (an
    // FP64 division costs about ten FP64-pipe operations, the Newton reciprocal four)
    const bool km = k > 0, kp = k < g.nz - 1;
    const long long a[7] = {c, cixw(g, i - 1, j, k), cixw(g, i + 1, j, k), cixw(g, i, j - 1, k), cixw(g, i, j + 1, k),
                            km ? c - g.nxy : c, kp ? c + g.nxy : c};
    double rr[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) rr[m] = rcp_d(__ldg(rho + a[m]));
    const double cxm = 0.5 * (hxm + h0) * hs * g.rdx, cxp = 0.5 * (h0 + hxp) * hs * g.rdx;
    const double cym = 0.5 * (hym + h0) * hs * g.rdy, cyp = 0.5 * (h0 + hyp) * hs * g.rdy;
    const double czm = km ? 0.5 * (__ldg(hk + c - g.nxy) + h0) * hs * g.rdzc[k] : 0.0;
    const double czp = kp ? 0.5 * (h0 + __ldg(hk + c + g.nxy)) * hs * g.rdzc[k + 1] : 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double v[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) v[m] = __ldg(rq.q[q] + a[m]) * rr[m];
        const double q0 = v[0];
        src.q[q][c] = (cxp * (v[2] - q0) - cxm * (q0 - v[1])) * g.rdx + (cyp * (v[4] - q0) - cym * (q0 - v[3])) * g.rdy
                    + (czp * (v[6] - q0) - czm * (q0 - v[5])) * g.rdzeta[k];
    }
}

// lateral relaxation zones (open x boundaries; Sec. 3.8 nudging toward boundary data, here the
// initial state): -tau_r(d) (S - S_ref) in every slow tendency and moisture source, d the distance
// of the point from the nearer x-edge (cells at their centres, x-faces at x = i dx)
__global__ void k_relax(Geo g, Phys ph, CF5 st, CF5 ref, F5 R, Q3 rq, Q3 rqref, Q3w qsrc) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), k = (int)(n / g.nxy);
    const double tc = relax_rate(ph, (i + 0.5) * g.dx), tf = relax_rate(ph, i * g.dx);
    if (k < g.nz) {
        R.r[n] -= tc * (st.r[n] - ref.r[n]);
        R.t[n] -= tc * (st.t[n] - ref.t[n]);
        R.u[n] -= tf * (st.u[n] - ref.u[n]);
        R.v[n] -= tc * (st.v[n] - ref.v[n]);
        if (ph.moist)
            for (int q = 0; q < 3; ++q) qsrc.q[q][n] -= tc * (rq.q[q][n] - rqref.q[q][n]);
    }
    if (k >= 1 && k < g.nz) R.w[n] -= tc * (st.w[n] - ref.w[n]);
}

// One time-split Kessler step after the RK3 step (Kessler 1969; Klemp & Wilhelmson 1978), the dry
// density unchanged, in two per-cell kernels (the rain fall needs only the rain before the fall, so
// no column recurrence is left):
//   k_kessler_fall: F = rho q_r V through each cell's bottom face, V = 36.34 (1e-3 rho q_r)^0.1346
//      (rho_0 / rho)^(1/2) m/s (the cgs form V = 3634 (rho q_r)^0.1346 (rho_0/rho)^(1/2) cm/s,
//      rho q_r in g/cm^3, rho_0 the base dry density at the ground);
//   k_kessler: the upwind fall step (what leaves the lowest cell adds F dt / rho_water to the
//      surface accumulation), then
//   2. autoconversion 1e-3 (q_c - 1e-3)^+ and accretion 2.2 q_c q_r^0.875 (1/s) move cloud to rain;
//   3. saturation adjustment in one linearised step (Soong & Ogura 1973) with the Tetens q_vs and
//      its slope q_vs 4098.17 / (T - 35.86)^2 at T = theta pi (pi from the moist EOS before the step);
//      rain evaporates min(dt E_r, (-s - q_c)^+, q_r), E_r = (1/rho) (1 - q_v/q_vs) C (rho q_r)^0.525
//      / (5.4e5 + 2.55e6 / (p q_vs)), C = 1.6 + 124.9 (rho q_r)^0.2046 (rho in g/cm^3, p in mb);
//      theta gains L_v / (c_p pi) (condensation - evaporation).
// Every quantity is applied as an increment of the conserved variables.
__global__ void k_kessler_fall(Geo g, const double *rho, const double *rqr, double *F) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny);
    const long long b0 = bix(g, i, j, 0);
    const double rho_sfc = g.rho0[b0] / (1.0 + g.qv0[b0]);
    const double r = rho[c], rr = rqr[c], qr = rr / r;
    F[c] = qr > 0.0 ? rr * (36.34 * pow(1.0e-3 * r * qr, 0.1346) * sqrt(rho_sfc / r)) : 0.0;
}
__global__ void k_kessler(Geo g, double dt, const double *F, double *rt, const double *rho, double *rqv,
                          double *rqc, double *rqr, double *precip) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    // 1. rain fall
    const double f_below = F[c], f_above = k + 1 < g.nz ? F[c + g.nxy] : 0.0;
    if (k == 0) precip[(long long)j * g.nx + i] += dt * f_below / RHOW;
    rqr[c] += dt * (f_above - f_below) * (g.terrain ? rHc(g, i, j, k) : g.rdzeta[k]);
    const double r = rho[c], th = rt[c] / r;
    const double qv = rqv[c] / r;
    double qc = rqc[c] / r, qr = rqr[c] / r;
    double p, pie;
    eos_pi(rt[c] * (1.0 + (RV / RD) * qv), p, pie);
    // 2. autoconversion and accretion
    double ar = fmax(1.0e-3 * (qc - 1.0e-3), 0.0);
    double cr = qr > 0.0 ? 2.2 * qc * pow(qr, 0.875) : 0.0;
    double prod = fmin(dt * (ar + cr), qc);
    qc -= prod;
    qr += prod;
    // 3. saturation adjustment and rain evaporation
    const double T = th * pie;
    const double es = 610.78 * exp(17.27 * (T - 273.16) / (T - 35.86));
    const double qvs = (RD / RV) * es / (p - es);
    const double sadj = (qv - qvs) / (1.0 + qvs * LV * 4098.17 / (CPD * (T - 35.86) * (T - 35.86)));
    double ern = 0.0;
    if (qr > 0.0 && qv < qvs) {
        const double rg = 1.0e-3 * r, X = rg * qr;
        const double C = 1.6 + 124.9 * pow(X, 0.2046);
        ern = dt * ((1.0 / rg) * (1.0 - qv / qvs) * C * pow(X, 0.525) / (5.4e5 + 2.55e6 / ((1.0e-2 * p) * qvs)));
    }
    ern = fmin(fmin(ern, fmax(-sadj - qc, 0.0)), qr);
    const double cond = sadj > -qc ? sadj : -qc;
    rt[c] += r * (LV / (CPD * pie) * (cond - ern));
    rqv[c] += r * (ern - cond);
    rqc[c] += r * (cond - prod);
    rqr[c] += r * (prod - ern);
}

// ------------------------------------------------------------------ slow tendencies

// WENO5-JS / WENO5-Z face value in FP64 (same candidates and weights as weno5<T>), arranged for
// GB300's FP64 rate: the middle candidate and the six indicator terms are formed from the four
// first differences of the stencil, the other candidates enter as differences from the middle
// one, the indicators (with eps) carry a common factor 12/13, and the normalisation of that
// correction takes one reciprocal (rcp1_d) instead of a division.
__device__ __forceinline__ double weno5_d(const double *q, bool left, int zflag) {
    double a, b, c, d, e;   // v_{-2}, v_{-1}, v_0, v_1, v_2 on the upwind side
    if (left) { a = q[0]; b = q[1]; c = q[2]; d = q[3]; e = q[4]; }
    else { a = q[5]; b = q[4]; c = q[3]; d = q[2]; e = q[1]; }
    const double d1 = a - b, d2 = b - c, d3 = c - d, d4 = d - e;
    const double p1 = fma(-1.0 / 6.0, d2, fma(-1.0 / 3.0, d3, c));  // (-b + 5c + 2d)/6
    const double t0 = d1 - d2, u0 = fma(-3.0, d2, d1);               // a - 2b + c, a - 4b + 3c
    const double t1 = d2 - d3, u1 = d2 + d3;                         // b - 2c + d, b - d
    const double t2 = d3 - d4, u2 = fma(3.0, d3, -d4);               // c - 2d + e, 3c - 4d + e
    // the other two candidates through their differences from p1: p0 - p1 = (t0 - t1)/3 and
    // p2 - p1 = (t1 - t2)/6, so that the value is p1 + (w0 (p0 - p1) + w2 (p2 - p1)) / sum w
    const double q0 = t0 - t1, q2 = t1 - t2;
    // eps + beta_r with beta_r = 13/12 t^2 + 1/4 u^2 and eps = 1e-6, all scaled by 12/13 (the
    // weights are homogeneous in eps + beta, so the scheme is unchanged): three FP64 operations
    constexpr double k3 = 3.0 / 13.0, eps = 1.0e-6 * (12.0 / 13.0);
    const double e0 = fma(t0, t0, fma(k3 * u0, u0, eps));
    const double e1 = fma(t1, t1, fma(k3 * u1, u1, eps));
    const double e2 = fma(t2, t2, fma(k3 * u2, u2, eps));
    if (zflag) {
        double tau = fabs(e0 - e2);   // |beta_0 - beta_2| (scaled)
        double w0 = 0.1 * (e0 + tau) * e1 * e2;
        double w1 = 0.6 * (e1 + tau) * e0 * e2;
        double w2 = 0.3 * (e2 + tau) * e0 * e1;
        double N = fma(w0, (1.0 / 3.0) * q0, w2 * ((1.0 / 6.0) * q2));
        return fma(N, rcp1_d(w0 + w1 + w2), p1);
    }
    // JS: w_r = d_r / (eps + b_r)^2 scaled by the product of all (eps + b)^2 and by 10/3, i.e.
    // (1/3) g0, 2 g1, g2 with g0 = (e1 e2)^2, g1 = (e0 e2)^2, g2 = (e0 e1)^2; the 1/3, 1/6 of the
    // differences fold into the constants
    const double f01 = e0 * e1, f02 = e0 * e2, f12 = e1 * e2;
    const double g0 = f12 * f12, g1 = f02 * f02, g2 = f01 * f01;
    const double D = fma(1.0 / 3.0, g0, fma(2.0, g1, g2));
    const double N = fma(g0 * (1.0 / 9.0), q0, g2 * ((1.0 / 6.0) * q2));
    return fma(N, rcp1_d(D), p1);
}

// face value of an advected scalar: WENO5-JS, WENO5-Z or the linear upwind-3 interpolant
__device__ __forceinline__ double scal_face_d(const double *q, bool left, int scheme) {
    return scheme == 3 ? upwind3_side<double>(q, left) : weno5_d(q, left, scheme == 1);
}

// theta fluxes through the left x-face, front y-face and bottom w-face of each cell (each face
// once): normal mass flux x WENO5(theta); walls carry none
__global__ void k_flux_theta(Geo g, Phys ph, Prep pr, const double *th, double *fx, double *fy, double *fz) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    double q[6];
    if (k < g.nz) {
        double mx = pr.mfx[n], my = pr.mfy[n];
        for (int m = 0; m < 6; ++m) q[m] = cval(g, th, i - 3 + m, j, k);
        fx[n] = mx * scal_face_d(q, upwind_left(mx), ph.scal_adv);
        for (int m = 0; m < 6; ++m) q[m] = cval(g, th, i, j - 3 + m, k);
        fy[n] = my * scal_face_d(q, upwind_left(my), ph.scal_adv);
    }
    if (k == 0 || k == g.nz) { fz[n] = 0.0; return; }
    double om = pr.rom[n];
    for (int m = 0; m < 6; ++m) q[m] = cval(g, th, i, j, k - 3 + m);
    fz[n] = om * scal_face_d(q, upwind_left(om), ph.scal_adv);
}

// continuity and potential temperature (Eq. con, Eq. theta): flux divergence / cell height
__global__ void k_rhs_cells(Geo g, Phys ph, CF5 st, Prep pr, const double *fx, const double *fy, const double *fz,
                            double *Rr, double *Rt) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    long long cxp = cixw(g, i + 1, j, k), cyp = cixw(g, i, j + 1, k), ckp = c + g.nxy;
    double rH = rHc(g, i, j, k);
    Rr[c] = -((pr.mfx[cxp] - pr.mfx[c]) * g.rdx + (pr.mfy[cyp] - pr.mfy[c]) * g.rdy + (pr.rom[ckp] - pr.rom[c])) * rH;
    double r = -((fx[cxp] - fx[c]) * g.rdx + (fy[cyp] - fy[c]) * g.rdy + (fz[ckp] - fz[c])) * rH;
    // Rayleigh damping of theta toward the base state theta0 (Sec. 3.7)
    if (ph.ray_fields & 8) r -= ray_rate(ph, zc(g, i, j, k)) * (st.t[c] - st.r[c] * g.th0[bix(g, i, j, k)]);
    Rt[c] = r;
}

// Advective momentum fluxes (reading R5), each computed once: the u-, v- and w-control volumes
// share every face with a neighbour, so the divergence kernels read two values per direction
// instead of evaluating both upwind-5 fluxes themselves.  One thread per (i, j, k), k = 0..nz.
#define CELL3D_W()                                                  \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;            \
    if (i >= g.nx) return;                                          \
    const int j = blockIdx.y, k = blockIdx.z;                       \
    const long long n = ((long long)k * g.ny + j) * g.nx + i;
// The advecting mass flux is the mean of two face mass fluxes; its 1/2 is folded into the
// interpolant's weights (exact), so adv below is their sum.
template <int mom3>
__device__ __forceinline__ double mom_face_h(const double *q, bool left) {
    return mom3 ? upwind3_side<double, 2>(q, left) : upwind5_side<double, 2>(q, left);
}
// u: x-flux at the cell centre (i,j,k), y-flux at the xy-edge (x-face i, y-face j), z-flux at the
// xz-edge (x-face i, w-face k; zero on the walls)
template <int mom3>
__global__ void k_flux_u(Geo g, Prep pr, double *fx, double *fy, double *fz) {
    CELL3D_W();
    double q[6];
    if (k < g.nz) {
        double adv = (__ldg(pr.mfx + n) + cval(g, pr.mfx, i + 1, j, k));
        for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.ux, i - 2 + m, j, k);
        fx[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
        adv = (cval(g, pr.mfy, i - 1, j, k) + __ldg(pr.mfy + n));
        for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.ux, i, j - 3 + m, k);
        fy[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
    }
    if (k == 0 || k == g.nz) { fz[n] = 0.0; return; }
    double adv = (__ldg(pr.rom + cixw(g, i - 1, j, k)) + __ldg(pr.rom + n));
    for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.ux, i, j, k - 3 + m);
    fz[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
}
// v: x-flux at the xy-edge (x-face i, y-face j), y-flux at the cell centre, z-flux at the yz-edge
template <int mom3>
__global__ void k_flux_v(Geo g, Prep pr, double *fx, double *fy, double *fz) {
    CELL3D_W();
    double q[6];
    if (k < g.nz) {
        double adv = (cval(g, pr.mfx, i, j - 1, k) + __ldg(pr.mfx + n));
        for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.vy, i - 3 + m, j, k);
        fx[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
        adv = (__ldg(pr.mfy + n) + cval(g, pr.mfy, i, j + 1, k));
        for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.vy, i, j - 2 + m, k);
        fy[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
    }
    if (k == 0 || k == g.nz) { fz[n] = 0.0; return; }
    double adv = (__ldg(pr.rom + cixw(g, i, j - 1, k)) + __ldg(pr.rom + n));
    for (int m = 0; m < 6; ++m) q[m] = cval(g, pr.vy, i, j, k - 3 + m);
    fz[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
}
// w: x-flux at the xz-edge (x-face i, w-face k), y-flux at the yz-edge (both [nz+1] planes, zero on
// the walls), z-flux at the cell centre (i,j,k) ([nz] planes)
template <int mom3>
__global__ void k_flux_w(Geo g, Prep pr, double *fx, double *fy, double *fz) {
    CELL3D_W();
    double q[6];
    if (k < g.nz) {
        double adv = (__ldg(pr.rom + n) + __ldg(pr.rom + n + g.nxy));
        for (int m = 0; m < 6; ++m) q[m] = wval(g, pr.wz, i, j, k - 2 + m);
        fz[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
    }
    if (k == 0 || k == g.nz) { fx[n] = 0.0; fy[n] = 0.0; return; }
    double adv = (cval(g, pr.mfx, i, j, k - 1) + __ldg(pr.mfx + n));
    for (int m = 0; m < 6; ++m) q[m] = __ldg(pr.wz + cixw(g, i - 3 + m, j, k));
    fx[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
    adv = (cval(g, pr.mfy, i, j, k - 1) + __ldg(pr.mfy + n));
    for (int m = 0; m < 6; ++m) q[m] = __ldg(pr.wz + cixw(g, i, j - 3 + m, k));
    fy[n] = adv * mom_face_h<mom3>(q, upwind_left(adv));
}

// x-momentum at x-face (i,j,k): upwind-5 advection (reading R5), terrain pressure gradient
// (App. B), Coriolis, -div(tau)
__global__ void k_rhs_u(Geo g, Phys ph, CF5 st, const double *pp, const double *fx, const double *fy,
                        const double *fz, double *Ru) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double div = (__ldg(fx + c) - __ldg(fx + cixw(g, i - 1, j, k))) * g.rdx
               + (__ldg(fy + cixw(g, i, j + 1, k)) - __ldg(fy + c)) * g.rdy + (__ldg(fz + c + g.nxy) - __ldg(fz + c));
    double r = -div * rHxf(g, i, j, k);
    // pressure gradient
    double px = (pp[c] - cval(g, pp, i - 1, j, k)) * g.rdx;
    if (g.terrain && g.nz > 1) {
        int kl = k == 0 ? 0 : k - 1, ku = k == g.nz - 1 ? g.nz - 1 : k + 1;
        double d0 = (cval(g, pp, i, j, ku) - cval(g, pp, i, j, kl)) * rdz2c(g, i, j, k);
        double d1 = (cval(g, pp, i - 1, j, ku) - cval(g, pp, i - 1, j, kl)) * rdz2c(g, i - 1, j, k);
        px -= hxi_x2(g, i, j, k) * (d0 + d1);
    }
    if (ph.moist) px /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i - 1, j, k), cval(g, st.r, i - 1, j, k)) + q_vc(ph, c, st.r[c]));
    r -= px;
    if (ph.f_cor != 0.0) {
        double rvx = 0.25 * (cval(g, st.v, i - 1, j, k) + cval(g, st.v, i, j, k) + cval(g, st.v, i - 1, j + 1, k) + cval(g, st.v, i, j + 1, k));
        double rhx = 0.5 * (cval(g, st.r, i - 1, j, k) + cval(g, st.r, i, j, k));
        r += ph.f_cor * (rvx - rhx * ph.v_g);
    }
    if (ph.ray_fields & 1) {   // Rayleigh damping toward u_g (Sec. 3.7)
        const double z = 0.5 * (zc(g, i - 1, j, k) + zc(g, i, j, k));
        r -= ray_rate(ph, z) * (st.u[c] - 0.5 * (cval(g, st.r, i - 1, j, k) + st.r[c]) * ph.u_g);
    }
    Ru[c] = r;
}

__global__ void k_rhs_v(Geo g, Phys ph, CF5 st, const double *pp, const double *fx, const double *fy,
                        const double *fz, double *Rv) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double div = (__ldg(fx + cixw(g, i + 1, j, k)) - __ldg(fx + c)) * g.rdx
               + (__ldg(fy + c) - __ldg(fy + cixw(g, i, j - 1, k))) * g.rdy + (__ldg(fz + c + g.nxy) - __ldg(fz + c));
    double r = -div * rHyf(g, i, j, k);
    double py = (pp[c] - cval(g, pp, i, j - 1, k)) * g.rdy;
    if (g.terrain && g.nz > 1) {
        int kl = k == 0 ? 0 : k - 1, ku = k == g.nz - 1 ? g.nz - 1 : k + 1;
        double d0 = (cval(g, pp, i, j, ku) - cval(g, pp, i, j, kl)) * rdz2c(g, i, j, k);
        double d1 = (cval(g, pp, i, j - 1, ku) - cval(g, pp, i, j - 1, kl)) * rdz2c(g, i, j - 1, k);
        py -= heta_y2(g, i, j, k) * (d0 + d1);
    }
    if (ph.moist) py /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i, j - 1, k), cval(g, st.r, i, j - 1, k)) + q_vc(ph, c, st.r[c]));
    r -= py;
    if (ph.f_cor != 0.0) {
        double rux = 0.25 * (cval(g, st.u, i, j - 1, k) + cval(g, st.u, i + 1, j - 1, k) + cval(g, st.u, i, j, k) + cval(g, st.u, i + 1, j, k));
        double rhy = 0.5 * (cval(g, st.r, i, j - 1, k) + cval(g, st.r, i, j, k));
        r -= ph.f_cor * (rux - rhy * ph.u_g);
    }
    if (ph.ray_fields & 2) {   // Rayleigh damping toward v_g (Sec. 3.7)
        const double z = 0.5 * (zc(g, i, j - 1, k) + zc(g, i, j, k));
        r -= ray_rate(ph, z) * (st.v[c] - 0.5 * (cval(g, st.r, i, j - 1, k) + st.r[c]) * ph.v_g);
    }
    Rv[c] = r;
}

// z-momentum at interior w-faces; boundary rows are zero
__global__ void k_rhs_w(Geo g, Phys ph, CF5 st, const double *pp, const double *fx, const double *fy,
                        const double *fz, double *Rw) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    if (k == 0 || k == g.nz) { Rw[n] = 0.0; return; }
    double div = (__ldg(fx + cixw(g, i + 1, j, k)) - __ldg(fx + n)) * g.rdx
               + (__ldg(fy + cixw(g, i, j + 1, k)) - __ldg(fy + n)) * g.rdy + (__ldg(fz + n) - __ldg(fz + n - g.nxy));
    double rdz = rdzcw(g, i, j, k);
    double r = -div * rdz;
    long long c = cix(g, i, j, k), cm = cix(g, i, j, k - 1);
    double b0 = g.rho0[bix(g, i, j, k - 1)], b1 = g.rho0[bix(g, i, j, k)];
    if (ph.anelastic) {
        // Sec. 2.2: B = rho0 g (theta - theta0) / theta0, the face mean of the two cells
        const double t0m = g.th0[bix(g, i, j, k - 1)], t0c = g.th0[bix(g, i, j, k)];
        const double Bm = b0 * ph.g * (st.t[cm] / st.r[cm] - t0m) / t0m;
        const double Bc = b1 * ph.g * (st.t[c] / st.r[c] - t0c) / t0c;
        r -= (pp[c] - pp[cm]) * rdz;
        r += 0.5 * (Bm + Bc);
    } else if (ph.moist) {
        // Eq. mom: (-dp'/dz + B) / (1 + q_v + q_c), B of the total density rho_d (1 + q_v + q_c + q_r)
        const double rm = st.r[cm] + (__ldg(ph.rqv + cm) + __ldg(ph.rqc + cm) + __ldg(ph.rqr + cm));
        const double rc = st.r[c] + (__ldg(ph.rqv + c) + __ldg(ph.rqc + c) + __ldg(ph.rqr + c));
        const double B = 0.5 * (-ph.g * (rm - b0) - ph.g * (rc - b1));
        const double f = 1.0 + 0.5 * (q_vc(ph, cm, st.r[cm]) + q_vc(ph, c, st.r[c]));
        // the dry path's order of operations (exact for f = 1: no water, the dry result)
        r -= (pp[c] - pp[cm]) * rdz / f;
        r += B / f;
    } else {
        r -= (pp[c] - pp[cm]) * rdz;
        r += 0.5 * (-ph.g * (st.r[cm] - b0) - ph.g * (st.r[c] - b1));
    }
    if (ph.ray_fields & 4) {   // Rayleigh damping toward w = 0 at the w-face height (Sec. 3.7)
        const double zw = g.zetac[k - 1] + 0.5 * g.dzeta[k - 1] + (g.terrain ? g.s[k] * g.hc[ij2(g, i, j)] : 0.0);
        r -= ray_rate(ph, zw) * st.w[n];
    }
    Rw[n] = r;
}

// ------------------------------------------------------------------ acoustic substeps (App. C)

// Per column: coefficients of the vertical system in Omega'' (reading R11) for this stage's
// dtau, and their LU factors (Thomas forward elimination without the right-hand side).  With
// E = dtau b2^2, the sums S_pi = pi_{k-1} + pi_k, S_rho = rho_{k-1} + rho_k and the w-face means
// thw of theta, the rows are
//   P = dtau (-C_pg + C_b pi_k / Theta_k),  Q = dtau (C_pg + C_b pi_{k-1} / Theta_{k-1}),
//   C_pg = gamma R_d (S_pi / 2) / dz_c,  C_b = g (R_d / c_v) (S_rho / 2) / S_pi,
//   a = (E Gg - E Q thw_{k-1/2}) / H_{k-1},  c = (E P thw_{k+1/2} - E Gg) / H_k,
//   b = 1 + thw_k (E Q / H_{k-1} - E P / H_k) + E Gg (1 / H_k - 1 / H_{k-1}),  Gg = dtau g / 2,
// with the stage constants (dtau, E, E Gg, the halves) formed on the host (TriK).  The w-face
// means of theta are carried up the column (each one is formed once) and stored for the substeps
// (THW, levels 0..nz, the wall faces taking the reflected cell's value).  Alongside: H theta^t / dx
// at x-faces and H theta^t / dy at y-faces (TX, TY) and dtau (-gamma R_d) (pi_{i-1} + pi_i) / 2 at
// x- and y-faces (PX, PY), the stage-fixed factors of the substeps' Theta'' fluxes and pressure
// gradients.
struct TriK {
    double E, EGg;    // dtau b2^2, E dtau g / 2
    double cpg;       // dtau gamma R_d / 2
    double kgb;       // dtau g (R_d / c_v) / 2
    double dpx;       // -dtau gamma R_d / 2
    double hrdx, hrdy;  // 1 / (2 dx), 1 / (2 dy): the face mean of theta and the substeps' 1/dx, 1/dy
};
__global__ void k_tri_build(Geo g, const double *rho, const double *rt, const double *pi, const double *th, TriK tk,
                            Tri tr, double *TX, double *TY, double *PX, double *PY, double *THW, Phys ph) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nxy) return;
    int i = (int)(n % g.nx), j = (int)(n / g.nx);
    const double E = tk.E, EGg = tk.EGg;
    double cp_prev = 0.0;
    double rrt_m = rcp_d(rt[cix(g, i, j, 0)]), rHm = rHc(g, i, j, 0);
    auto face_factors = [&](int k) {
        long long c = cix(g, i, j, k);
        double thc = th[c], pic = pi[c];
        TX[c] = Hx(g, i, j, k) * (tk.hrdx * (cval(g, th, i - 1, j, k) + thc));
        TY[c] = Hy(g, i, j, k) * (tk.hrdy * (cval(g, th, i, j - 1, k) + thc));
        PX[c] = tk.dpx * (cval(g, pi, i - 1, j, k) + pic);
        PY[c] = tk.dpx * (cval(g, pi, i, j - 1, k) + pic);
        if (ph.moist) {   // App. C: gamma R_d pi^t / (1 + q_v^t + q_c^t) at the face
            const double qc0 = q_vc(ph, c, rho[c]);
            PX[c] /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i - 1, j, k), cval(g, rho, i - 1, j, k)) + qc0);
            PY[c] /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i, j - 1, k), cval(g, rho, i, j - 1, k)) + qc0);
        }
    };
    face_factors(0);
    double th_m = th[cix(g, i, j, 0)];
    double thw_m = th_m;                                 // the wall reflection: theta_{-1} = theta_0
    double thw_k = 0.5 * (th_m + cval(g, th, i, j, 1));
    THW[cix(g, i, j, 0)] = th_m;
    THW[cix(g, i, j, g.nz)] = th[cix(g, i, j, g.nz - 1)];
    for (int k = 1; k < g.nz; ++k) {
        face_factors(k);
        long long c = cix(g, i, j, k), cm = c - g.nxy, w = c;
        THW[w] = thw_k;
        double thw_p = 0.5 * (th[c] + cval(g, th, i, j, k + 1));
        double pic = pi[c], pim = pi[cm];
        double Spi = pim + pic;
        double Cpg = tk.cpg * Spi * rdzcw(g, i, j, k);
        double Cb = tk.kgb * (rho[cm] + rho[c]) * rcp_d(Spi);
        if (ph.moist) {
            // App. C: the pressure term over 1 + q_v + q_c, the Theta'' buoyancy times rho_d / rho_m
            Cpg /= 1.0 + 0.5 * (q_vc(ph, cm, rho[cm]) + q_vc(ph, c, rho[c]));
            Cb /= 1.0 + 0.5 * (q_t(ph, cm, rho[cm]) + q_t(ph, c, rho[c]));
        }
        double rrt_c = rcp_d(rt[c]), rHk = rHc(g, i, j, k);
        double P = fma(Cb * pic, rrt_c, -Cpg);
        double Q = fma(Cb * pim, rrt_m, Cpg);
        double Pe = E * P, Qe = E * Q;
        double a = fma(-Qe, thw_m, EGg) * rHm;
        double cc = fma(Pe, thw_p, -EGg) * rHk;
        double b = fma(thw_k, fma(-Pe, rHk, Qe * rHm), 1.0);
        b = fma(EGg, rHk - rHm, b);
        double im = rcp_d(fma(-a, cp_prev, b));
        double cpk = cc * im;
        tr.a[w] = a; tr.cp[w] = cpk; tr.im[w] = im; tr.P[w] = P; tr.Q[w] = Q;
        cp_prev = cpk;
        rrt_m = rrt_c;
        rHm = rHk;
        thw_m = thw_k;
        thw_k = thw_p;
    }
}

// The same system for grids with few columns (a 2D slab has a few thousand): one warp per column.
// The lanes form every level's face factors, w-face theta and row coefficients at once (the same
// operands and operations as k_tri_build), then lane 0 runs only the LU recurrence
// im_k = 1 / (b_k - a_k cp_{k-1}), cp_k = c_k im_k over shared memory.  Bit-identical to
// k_tri_build.  nz <= TRIW_NZ.
constexpr int TRIW_WARPS = 4, TRIW_NZ = 256;
__global__ void __launch_bounds__(32 * TRIW_WARPS) k_tri_build_warp(Geo g, const double *rho, const double *rt,
                                                                     const double *pi, const double *th, TriK tk,
                                                                     Tri tr, double *TX, double *TY, double *PX,
                                                                     double *PY, double *THW, Phys ph) {
    __shared__ double sb[TRIW_WARPS][TRIW_NZ], sc[TRIW_WARPS][TRIW_NZ], sa[TRIW_WARPS][TRIW_NZ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n = (long long)blockIdx.x * TRIW_WARPS + warp;
    if (n >= g.nxy) return;
    const int i = (int)(n % g.nx), j = (int)(n / g.nx), nz = g.nz;
    const double E = tk.E, EGg = tk.EGg;
    for (int k = lane; k < nz; k += 32) {
        long long c = cix(g, i, j, k);
        double thc = th[c], pic = pi[c];
        TX[c] = Hx(g, i, j, k) * (tk.hrdx * (cval(g, th, i - 1, j, k) + thc));
        TY[c] = Hy(g, i, j, k) * (tk.hrdy * (cval(g, th, i, j - 1, k) + thc));
        PX[c] = tk.dpx * (cval(g, pi, i - 1, j, k) + pic);
        PY[c] = tk.dpx * (cval(g, pi, i, j - 1, k) + pic);
        if (ph.moist) {
            const double qc0 = q_vc(ph, c, rho[c]);
            PX[c] /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i - 1, j, k), cval(g, rho, i - 1, j, k)) + qc0);
            PY[c] /= 1.0 + 0.5 * (q_vc(ph, cixw(g, i, j - 1, k), cval(g, rho, i, j - 1, k)) + qc0);
        }
        // w-face theta below cell k (the wall reflection at k = 0) and, for the top cell, at the lid
        THW[c] = k == 0 ? thc : 0.5 * (th[c - g.nxy] + thc);
        if (k == nz - 1) THW[cix(g, i, j, nz)] = thc;
    }
    for (int k = 1 + lane; k < nz; k += 32) {
        long long c = cix(g, i, j, k), cm = c - g.nxy, w = c;
        const double thw_m = k == 1 ? th[cm] : 0.5 * (th[cm - g.nxy] + th[cm]);
        const double thw_k = 0.5 * (th[cm] + th[c]);
        const double thw_p = 0.5 * (th[c] + cval(g, th, i, j, k + 1));
        double pic = pi[c], pim = pi[cm];
        double Spi = pim + pic;
        double Cpg = tk.cpg * Spi * rdzcw(g, i, j, k);
        double Cb = tk.kgb * (rho[cm] + rho[c]) * rcp_d(Spi);
        if (ph.moist) {
            Cpg /= 1.0 + 0.5 * (q_vc(ph, cm, rho[cm]) + q_vc(ph, c, rho[c]));
            Cb /= 1.0 + 0.5 * (q_t(ph, cm, rho[cm]) + q_t(ph, c, rho[c]));
        }
        double rrt_c = rcp_d(rt[c]), rrt_m = rcp_d(rt[cm]), rHk = rHc(g, i, j, k), rHm = rHc(g, i, j, k - 1);
        double P = fma(Cb * pic, rrt_c, -Cpg);
        double Q = fma(Cb * pim, rrt_m, Cpg);
        double Pe = E * P, Qe = E * Q;
        double a = fma(-Qe, thw_m, EGg) * rHm;
        double cc = fma(Pe, thw_p, -EGg) * rHk;
        double b = fma(thw_k, fma(-Pe, rHk, Qe * rHm), 1.0);
        b = fma(EGg, rHk - rHm, b);
        tr.a[w] = a; tr.P[w] = P; tr.Q[w] = Q;
        sa[warp][k] = a; sb[warp][k] = b; sc[warp][k] = cc;
    }
    __syncwarp();
    if (lane == 0) {
        double cp_prev = 0.0;
        for (int k = 1; k < nz; ++k) {
            const long long w = cix(g, i, j, k);
            double im = rcp_d(fma(-sa[warp][k], cp_prev, sb[warp][k]));
            double cpk = sc[warp][k] * im;
            tr.cp[w] = cpk; tr.im[w] = im;
            cp_prev = cpk;
        }
    }
}

// horizontal momenta: Delta U'' = dtau (-gamma R_d pi^t (dTheta~/dxi - h_xi/h_zeta dTheta~/dzeta) + R_U),
// Theta~ = Theta'' + beta_d (Theta'' - Theta''_prev) (reading R10), which the previous vertical
// solve (or the stage start, where Theta~ = Theta'') left in Tt.  PX, PY hold the stage's
// dtau (-gamma R_d) pi^t at x- and y-faces.
__global__ void k_sub_horiz(Geo g, const double *PX, const double *PY, const double *Tt, const double *Ru,
                            const double *Rv, double *Xu, double *Xv, double dtau) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double t0 = __ldg(Tt + c);
    double gx = (t0 - cval(g, Tt, i - 1, j, k)) * g.rdx;
    double gy = (t0 - cval(g, Tt, i, j - 1, k)) * g.rdy;
    if (g.terrain && g.nz > 1) {
        int kl = k == 0 ? 0 : k - 1, ku = k == g.nz - 1 ? g.nz - 1 : k + 1;
        double dc = (cval(g, Tt, i, j, ku) - cval(g, Tt, i, j, kl)) * rdz2c(g, i, j, k);
        double dxm = (cval(g, Tt, i - 1, j, ku) - cval(g, Tt, i - 1, j, kl)) * rdz2c(g, i - 1, j, k);
        double dym = (cval(g, Tt, i, j - 1, ku) - cval(g, Tt, i, j - 1, kl)) * rdz2c(g, i, j - 1, k);
        gx -= hxi_x2(g, i, j, k) * (dc + dxm);
        gy -= heta_y2(g, i, j, k) * (dc + dym);
    }
    Xu[c] = fma(dtau, Ru[c], fma(PX[c], gx, Xu[c]));
    Xv[c] = fma(dtau, Rv[c], fma(PY[c], gy, Xv[c]));
}

// Vertical acoustic update (App. C rows 3-5) in three kernels.  Part 1, one thread per cell:
// explicit Theta*, rho* from the new U'', V'' divergence and the beta_1 part of the old Omega''
// flux; the beta-weighted X0 = b1 Theta''^tau + b2 Theta*, Y0 = b1 rho''^tau + b2 rho* of the
// Omega'' rows; and, at the cell's bottom w-face, W'' - (metric shift) + dtau R_W.  TX, TY hold
// H theta^t / dx at x-faces and H theta^t / dy at y-faces for this stage.  Theta''^tau is kept in
// Tt.
__global__ void k_sub_expl(Geo g, Phys ph, const double *thw, const double *TX, const double *TY, const double *Rr,
                           const double *Rt, const double *Rw, F5 x, const double *Om, double *Tt, double *X0,
                           double *Y0, double *Ash, double *msx, double *msy, double *msz, double dtau) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y, k = blockIdx.z, nz = g.nz;
    const long long nxy = g.nxy;
    const long long c = ((long long)k * g.ny + j) * g.nx + i;
    const long long oxp = i + 1 < g.nx ? 1 : 1 - g.nx;
    const long long oyp = j + 1 < g.ny ? (long long)g.nx : (long long)g.nx - nxy;
    const double b1 = ph.b1, b2 = ph.b2;
    double om_k = k >= 1 ? Om[c] : 0.0;
    double om_p = k + 1 < nz ? Om[c + nxy] : 0.0;
    // theta^t at the lower and upper w-faces
    double tw_k = thw[c], tw_p = thw[c + nxy];
    double Uc = x.u[c], Up = x.u[c + oxp], Vc = x.v[c], Vp = x.v[c + oyp];
    double divM = (Hx(g, i + 1, j, k) * Up - Hx(g, i, j, k) * Uc) * g.rdx
                + (Hy(g, i, j + 1, k) * Vp - Hy(g, i, j, k) * Vc) * g.rdy;
    double divT = (__ldg(TX + c + oxp) * Up - __ldg(TX + c) * Uc) + (__ldg(TY + c + oyp) * Vp - __ldg(TY + c) * Vc);
    double rH = rHc(g, i, j, k);
    double xt = x.t[c], xr = x.r[c];
    double Ts = xt + dtau * ((-divT - b1 * (om_p * tw_p - om_k * tw_k)) * rH + Rt[c]);
    double Rs = xr + dtau * ((-divM - b1 * (om_p - om_k)) * rH + Rr[c]);
    Tt[c] = xt;
    x.t[c] = Ts;
    x.r[c] = Rs;
    X0[c] = b1 * xt + b2 * Ts;
    Y0[c] = b1 * xr + b2 * Rs;
    if (k >= 1) {
        double A = 0.0;
        if (g.terrain) {
            A = metric_shift(g, x.u, x.v, i, j, k);
            Ash[c] = A;
        }
        x.w[c] = x.w[c] - A + dtau * Rw[c];
    }
    if (msx) {   // passive scalar: this substep's perturbation mass fluxes that advance rho''
        msx[c] += Hx(g, i, j, k) * Uc;
        msy[c] += Hy(g, i, j, k) * Vc;
        if (k >= 1) msz[c] += b1 * om_k;
    }
}

// Part 2, one thread per column: the Omega'' rows' right-hand side, forward substitution with the
// stage LU factors (d' held in Om) and back substitution.  Only the recurrences are serial; the
// operands of SB levels are loaded ahead of each stretch of the recurrence, so a thread keeps
// 7 SB loads in flight (the columns alone do not fill the GPU with warps).
constexpr int SB = 8;
__global__ void __launch_bounds__(128) k_sub_col(int nz, long long nxy, const double *__restrict__ ta,
                                                 const double *__restrict__ tcp, const double *__restrict__ tim,
                                                 const double *__restrict__ tP, const double *__restrict__ tQ,
                                                 const double *__restrict__ X0, const double *__restrict__ Y0,
                                                 double *__restrict__ W, double *__restrict__ Om, double Gg) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= nxy) return;
    double dpm = 0.0;
    double X0m = X0[n], Y0m = Y0[n];
    auto fwd = [&](long long c, double X0c, double Y0c, double Wc, double Pc, double Qc, double ac, double imc) {
        double rhs = Wc + Pc * X0c + Qc * X0m - Gg * (Y0c + Y0m);
        double dp = (rhs - ac * dpm) * imc;
        Om[c] = dp;
        dpm = dp;
        X0m = X0c; Y0m = Y0c;
    };
    int k = 1;
    for (; k + SB <= nz; k += SB) {
        double xv[SB], yv[SB], wv[SB], pv[SB], qv[SB], av[SB], iv[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            long long c = n + (long long)(k + u) * nxy;
            xv[u] = X0[c]; yv[u] = Y0[c]; wv[u] = W[c]; pv[u] = tP[c]; qv[u] = tQ[c]; av[u] = ta[c]; iv[u] = tim[c];
        }
#pragma unroll
        for (int u = 0; u < SB; ++u)
            fwd(n + (long long)(k + u) * nxy, xv[u], yv[u], wv[u], pv[u], qv[u], av[u], iv[u]);
    }
    for (; k < nz; ++k) {
        long long c = n + (long long)k * nxy;
        fwd(c, X0[c], Y0[c], W[c], tP[c], tQ[c], ta[c], tim[c]);
    }
    long long top = n + nz * nxy;
    W[top] = 0.0;
    Om[top] = 0.0;
    double om_up = 0.0;
    k = nz - 1;
    for (; k - SB >= 0; k -= SB) {   // levels k, k - 1, ..., k - SB + 1 (all >= 1)
        double ov[SB], cv[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            long long c = n + (long long)(k - u) * nxy;
            ov[u] = Om[c]; cv[u] = tcp[c];
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            double om = ov[u] - cv[u] * om_up;
            Om[n + (long long)(k - u) * nxy] = om;
            om_up = om;
        }
    }
    for (; k >= 1; --k) {
        long long c = n + (long long)k * nxy;
        double om = Om[c] - tcp[c] * om_up;
        Om[c] = om;
        om_up = om;
    }
    Om[n] = 0.0;
}

// Part 2 for grids with few columns: one warp per column.  The forward substitution
// d'_k = (r_k - a_k d'_{k-1}) / m_k and the back substitution Omega_k = d'_k - c'_k Omega_{k+1} are
// affine in their incoming value, so each lane takes a segment of at most SCW rows, composes its
// segment's map x -> A x + B, a warp scan (shuffles) of the composed maps gives every lane its
// incoming value, and the lane recomputes its rows with the same formulas as k_sub_col (the rows'
// operands stay in registers).  The values differ from k_sub_col's at rounding level only (the
// incoming values come through the composed maps).  nz <= 32 SCW + 1.
constexpr int SCW = 8;
__device__ __forceinline__ void affine_compose(double &A, double &B, double A2, double B2) {
    // (A2, B2) after (A, B): x -> A2 (A x + B) + B2
    B = fma(A2, B, B2);
    A = A2 * A;
}
__global__ void __launch_bounds__(128) k_sub_col_warp(int nz, long long nxy, const double *__restrict__ ta,
                                                      const double *__restrict__ tcp, const double *__restrict__ tim,
                                                      const double *__restrict__ tP, const double *__restrict__ tQ,
                                                      const double *__restrict__ X0, const double *__restrict__ Y0,
                                                      double *__restrict__ W, double *__restrict__ Om, double Gg) {
    const int lane = threadIdx.x & 31;
    const long long n = (long long)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (n >= nxy) return;
    const int rows = nz - 1, chunk = (rows + 31) / 32;
    const int k0 = 1 + lane * chunk, k1 = min(k0 + chunk, nz);
    double rv[SCW], av[SCW], iv[SCW], cv[SCW], dv[SCW];
    // the rows' right-hand sides and factors; the segment's forward map
    double A = 1.0, B = 0.0;
    for (int u = 0; u < SCW; ++u) {
        const int k = k0 + u;
        if (k >= k1) break;
        const long long c = n + (long long)k * nxy, cm = c - nxy;
        rv[u] = W[c] + tP[c] * X0[c] + tQ[c] * X0[cm] - Gg * (Y0[c] + Y0[cm]);
        av[u] = ta[c];
        iv[u] = tim[c];
        cv[u] = tcp[c];
        affine_compose(A, B, -av[u] * iv[u], rv[u] * iv[u]);
    }
    // exclusive scan over the lanes (lane 0 starts from d'_0 = 0)
    double sA = A, sB = B;
    for (int o = 1; o < 32; o <<= 1) {
        const double pA = __shfl_up_sync(0xffffffffu, sA, o), pB = __shfl_up_sync(0xffffffffu, sB, o);
        if (lane >= o) { double a2 = sA, b2 = sB; sA = pA; sB = pB; affine_compose(sA, sB, a2, b2); }
    }
    double din = __shfl_up_sync(0xffffffffu, sB, 1);   // the composed maps applied to 0
    if (lane == 0) din = 0.0;
    double dpm = din;
    for (int u = 0; u < SCW; ++u) {
        const int k = k0 + u;
        if (k >= k1) break;
        const double dp = (rv[u] - av[u] * dpm) * iv[u];
        dv[u] = dp;
        dpm = dp;
    }
    // back substitution from the lid (Omega_nz = 0): the segment's map from above, a reverse scan
    A = 1.0; B = 0.0;
    for (int u = SCW - 1; u >= 0; --u) {
        const int k = k0 + u;
        if (k >= k1) continue;
        affine_compose(A, B, -cv[u], dv[u]);
    }
    sA = A; sB = B;
    for (int o = 1; o < 32; o <<= 1) {
        const double pA = __shfl_down_sync(0xffffffffu, sA, o), pB = __shfl_down_sync(0xffffffffu, sB, o);
        if (lane + o < 32) { double a2 = sA, b2 = sB; sA = pA; sB = pB; affine_compose(sA, sB, a2, b2); }
    }
    double oin = __shfl_down_sync(0xffffffffu, sB, 1);
    if (lane == 31) oin = 0.0;
    double om_up = oin;
    for (int u = SCW - 1; u >= 0; --u) {
        const int k = k0 + u;
        if (k >= k1) continue;
        const double om = dv[u] - cv[u] * om_up;
        Om[n + (long long)k * nxy] = om;
        om_up = om;
    }
    if (lane == 0) {
        const long long top = n + (long long)nz * nxy;
        W[top] = 0.0;
        Om[top] = 0.0;
        Om[n] = 0.0;
    }
}

// Part 3, one thread per cell: Theta'', rho'' from the new Omega'' (beta_2 part), Theta~ of the
// next substep, and W'' = Omega'' + metric shift at the cell's bottom w-face.
__global__ void k_sub_fin(Geo g, Phys ph, const double *thw, const double *Om, const double *Ash, F5 x, double *Tt,
                          double *msz, double dtb2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long c = ((long long)k * g.ny + j) * g.nx + i;
    const double b2 = ph.b2, bd = ph.beta_d;
    double om = Om[c], om_up = Om[c + g.nxy];
    double thw_k = thw[c], thw_p = thw[c + g.nxy];
    double db = dtb2 * rHc(g, i, j, k);   // dtb2 = dtau b2
    double xt = x.t[c] - db * (om_up * thw_p - om * thw_k);
    x.t[c] = xt;
    x.r[c] = x.r[c] - db * (om_up - om);
    double told = Tt[c];
    Tt[c] = xt + bd * (xt - told);
    double A = 0.0;
    if (g.terrain) A = k >= 1 ? Ash[c] : metric_shift(g, x.u, x.v, i, j, 0);
    x.w[c] = om + A;
    if (msz && k >= 1) msz[c] += b2 * om;
}

// ------------------------------------------------------------------ passive scalar (Sec. 3.1)
// After a stage's substeps: rho phi^(s) = rho phi^n + alpha_s dt R_phi(phi^t), the advective
// fluxes taking the stage-averaged normal momenta that advanced rho (the stage mass flux plus
// the mean of the substeps' perturbation fluxes, summed in msx, msy, msz), so that phi = 1 stays
// 1.  phi^t is interpolated like theta (WENO5).
__global__ void k_tracer_phi(Geo g, const double *rphi, const double *rho, double *phi) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    phi[c] = rphi[c] * rcp_d(rho[c]);
}
__global__ void k_tracer_flux(Geo g, Phys ph, const double *ru, const double *rv, const double *rom,
                              const double *phi, const double *msx, const double *msy, const double *msz,
                              double rns, double *fx, double *fy, double *fz) {
    CELL3D_W();
    double q[6];
    if (k < g.nz) {
        double mx = Hx(g, i, j, k) * ru[n] + msx[n] * rns;
        for (int m = 0; m < 6; ++m) q[m] = cval(g, phi, i - 3 + m, j, k);
        fx[n] = mx * scal_face_d(q, upwind_left(mx), ph.scal_adv);
        double my = Hy(g, i, j, k) * rv[n] + msy[n] * rns;
        for (int m = 0; m < 6; ++m) q[m] = cval(g, phi, i, j - 3 + m, k);
        fy[n] = my * scal_face_d(q, upwind_left(my), ph.scal_adv);
    }
    if (k == 0 || k == g.nz) { fz[n] = 0.0; return; }
    double mz = rom[n] + msz[n] * rns;
    for (int m = 0; m < 6; ++m) q[m] = cval(g, phi, i, j, k - 3 + m);
    fz[n] = mz * scal_face_d(q, upwind_left(mz), ph.scal_adv);
}
// rho q^(s) = rho q^n + alpha dt (-div F / H + src) for a transported scalar; src (may be null)
// is the scalar's own source at the stage state; clip = 1 keeps rho q >= 0 (the SGS energy)
__global__ void k_tracer_update(Geo g, const double *snphi, const double *fx, const double *fy, const double *fz,
                                const double *src, int clip, double adt, double *rphi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long c = ((long long)k * g.ny + j) * g.nx + i;
    double div = (fx[cixw(g, i + 1, j, k)] - fx[c]) * g.rdx + (fy[cixw(g, i, j + 1, k)] - fy[c]) * g.rdy
               + (fz[c + g.nxy] - fz[c]);
    double t = -div * rHc(g, i, j, k);
    if (src) t += src[c];
    const double v = snphi[c] + adt * t;
    rphi[c] = (clip && v < 0.0) ? 0.0 : v;
}
__global__ void k_tracer_init(Geo g, const double *rho, const double *phi0, double *rphi) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    rphi[c] = rho[c] * phi0[c];
}

__global__ void k_stage_end(Geo g, F5 st, CF5 x) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    if (n < g.nc) {
        st.r[n] += x.r[n];
        st.t[n] += x.t[n];
        st.u[n] += x.u[n];
        st.v[n] += x.v[n];
    }
    st.w[n] += x.w[n];
}

// no-substep stage (Sec. 3.1): S^(s) = S^n + alpha dt R(S^t)
__global__ void k_stage_nosub(Geo g, F5 st, CF5 sn, CF5 R, double adt) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    if (n < g.nc) {
        st.r[n] = sn.r[n] + adt * R.r[n];
        st.t[n] = sn.t[n] + adt * R.t[n];
        st.u[n] = sn.u[n] + adt * R.u[n];
        st.v[n] = sn.v[n] + adt * R.v[n];
    }
    st.w[n] = sn.w[n] + adt * R.w[n];
}

// ------------------------------------------------------------------ diagnostics
// Fixed-shape, fixed-order reductions (deterministic): DIAG_BLOCKS x 256 threads, each thread
// a strided range, block tree reduction, then one block over the partials.
constexpr int DIAG_BLOCKS = 512;
__global__ void k_diag_partial(Geo g, CF5 st, double *part) {
    __shared__ double sm[256], sw[256], smn[256], smx[256], scfl[256], snf[256];
    int t = threadIdx.x;
    double mass = 0.0, wmax = 0.0, tmn = 1e300, tmx = -1e300, cfl = 0.0, nf = 0.0;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = blockIdx.x * (long long)blockDim.x + t; n < g.nw; n += stride) {
        int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
        if (k < g.nz) {
            double r = st.r[n], rt = st.t[n];
            mass += r * Hc(g, i, j, k) * g.dx * g.dy;
            double th = rt / r;
            tmn = fmin(tmn, th); tmx = fmax(tmx, th);
            double u = st.u[n] / (0.5 * (cval(g, st.r, i - 1, j, k) + r));
            double p, pie;
            eos_pi(rt, p, pie);
            double cs = sqrt(GAMMA * p / r);
            cfl = fmax(cfl, (fabs(u) + cs) * g.rdx);
            if (!isfinite(r) || !isfinite(rt) || !isfinite(st.u[n]) || !isfinite(st.v[n])) nf = 1.0;
        }
        double w = st.w[n];
        if (!isfinite(w)) nf = 1.0;
        if (k > 0 && k < g.nz) {
            double rb = 0.5 * (st.r[cix(g, i, j, k - 1)] + st.r[cix(g, i, j, k)]);
            wmax = fmax(wmax, fabs(w / rb));
        }
    }
    sm[t] = mass; sw[t] = wmax; smn[t] = tmn; smx[t] = tmx; scfl[t] = cfl; snf[t] = nf;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sm[t] += sm[t + s];
            sw[t] = fmax(sw[t], sw[t + s]);
            smn[t] = fmin(smn[t], smn[t + s]);
            smx[t] = fmax(smx[t], smx[t + s]);
            scfl[t] = fmax(scfl[t], scfl[t + s]);
            snf[t] = fmax(snf[t], snf[t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        double *p = part + 6 * blockIdx.x;
        p[0] = sm[0]; p[1] = sw[0]; p[2] = smn[0]; p[3] = smx[0]; p[4] = scfl[0]; p[5] = snf[0];
    }
}
__global__ void k_diag_final(const double *part, int nb, double dt, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mass = 0.0, wmax = 0.0, tmn = 1e300, tmx = -1e300, cfl = 0.0, nf = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double *p = part + 6 * b;
        mass += p[0]; wmax = fmax(wmax, p[1]); tmn = fmin(tmn, p[2]); tmx = fmax(tmx, p[3]);
        cfl = fmax(cfl, p[4]); nf = fmax(nf, p[5]);
    }
    out[0] = mass; out[1] = wmax; out[2] = tmn; out[3] = tmx; out[4] = cfl * dt; out[5] = nf;
}

// ------------------------------------------------------------------ dtype conversion
__global__ void k_f32_to_f64(const float *src, double *dst, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) dst[t] = (double)src[t];
}
__global__ void k_f64_to_f32(const double *src, float *dst, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) dst[t] = (float)src[t];
}

// ------------------------------------------------------------------ launchers
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
constexpr int BS = 256;

// the column kernels with one warp per column: -1 (default) below 2^15 columns, 0 never, 1 always
// (nz <= 256); set per step enqueue by the handle (erf_set_option ERF_OPT_WARP_COLUMNS)
// threads per block of the one-thread-per-column kernels: each thread runs a whole column, so an
// SM's time is its number of columns; with few columns (a few blocks per SM) small blocks spread
// them evenly over the SMs (128-thread blocks leave some SMs a whole block more than others)
static int col_block(const Geo &g) { return g.nxy <= (1LL << 18) ? 32 : 128; }
static thread_local int g_warp_columns = -1;
void set_warp_columns(int mode) { g_warp_columns = mode; }
static bool warp_columns(const Geo &g) {
    if (g.nz > TRIW_NZ) return false;
    if (g_warp_columns >= 0) return g_warp_columns == 1;
    return g.nxy < (1LL << 15);
}

// Optional per-launch event timing (profiling mode, never inside a graph capture).
static thread_local ProfSink *g_prof = nullptr;
void set_profiler(ProfSink *p) { g_prof = p; }
ProfSink *current_profiler() { return g_prof; }
struct ProfScope {
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(const char *n, cudaStream_t st) : s(st), name(n) {
        if (g_prof) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope() {
        if (g_prof) {
            cudaEventRecord(b, s);
            g_prof->add(name, a, b);
        }
    }
};
#define LAUNCH(name, s, ...)              \
    do {                                  \
        ProfScope _ps(name, s);           \
        __VA_ARGS__;                      \
    } while (0)

void launch_terrain(const Geo &g, const double *hn, double *hc, double *hxf, double *hyf, double *gxh,
                    double *gyh, double *g4xq, double *g4yq, cudaStream_t s) {
    LAUNCH("terrain_avg", s, k_terrain_avg<<<nblk(g.nxy, BS), BS, 0, s>>>(g, hn, hc, hxf, hyf));
    LAUNCH("terrain_grad", s, k_terrain_grad<<<nblk(g.nxy, BS), BS, 0, s>>>(g, hc, gxh, gyh, g4xq, g4yq));
}
void launch_terrain_recip(const Geo &g, double *Hx3, double *Hy3, double *rH3, double *rHx3, double *rHy3,
                          double *rdzw3, double *rdz2,
                          cudaStream_t s) {
    LAUNCH("terrain_recip", s, k_terrain_recip<<<nblk(g.nc, BS), BS, 0, s>>>(g, Hx3, Hy3, rH3, rHx3, rHy3, rdzw3, rdz2));
}
void launch_base_state(const Geo &g, int n_knots, const double *kz, const double *kt, double theta_s, double N,
                       double p_s, double grav, double *rho0, double *th0, double *p0, cudaStream_t s,
                       int n_qknots, const double *qz, const double *qk, double *qv0) {
    ThetaProfile tp{n_knots, kz, kt, theta_s, N, grav};
    QvProfile qp{n_qknots, qz, qk};
    long long ncol = g.terrain ? g.nxy : 1;
    LAUNCH("base_state", s, k_base_state<<<nblk(ncol, 128), 128, 0, s>>>(g, tp, qp, p_s, grav, rho0, th0, p0, qv0));
}
void launch_set_initial_moist(const Geo &g, const double *dth, const double *qv, const double *u, const double *v,
                              const double *w, double *rho, double *rt, double *ru, double *rv, double *rw,
                              double *rqv, double *rqc, double *rqr, cudaStream_t s) {
    LAUNCH("init_cells", s, k_init_cells_moist<<<nblk(g.nc, BS), BS, 0, s>>>(g, dth, qv, rho, rt, rqv, rqc, rqr));
    LAUNCH("init_faces", s, k_init_faces<<<nblk(g.nw, BS), BS, 0, s>>>(g, u, v, w, rho, ru, rv, rw));
    LAUNCH("wall_bc", s, k_wall_bc<<<nblk(g.nxy, BS), BS, 0, s>>>(g, ru, rv, rw));
}
void launch_kessler(const Geo &g, double dt, double *rt, const double *rho, double *rqv, double *rqc, double *rqr,
                    double *precip, double *fscratch, cudaStream_t s) {
    LAUNCH("kessler_fall", s, k_kessler_fall<<<nblk(g.nc, BS), BS, 0, s>>>(g, rho, rqr, fscratch));
    LAUNCH("kessler", s, k_kessler<<<nblk(g.nc, BS), BS, 0, s>>>(g, dt, fscratch, rt, rho, rqv, rqc, rqr, precip));
}
void launch_set_initial(const Geo &g, const double *dth, const double *u, const double *v, const double *w,
                        double *rho, double *rt, double *ru, double *rv, double *rw, cudaStream_t s) {
    LAUNCH("init_cells", s, k_init_cells<<<nblk(g.nc, BS), BS, 0, s>>>(g, dth, rho, rt));
    LAUNCH("init_faces", s, k_init_faces<<<nblk(g.nw, BS), BS, 0, s>>>(g, u, v, w, rho, ru, rv, rw));
    LAUNCH("wall_bc", s, k_wall_bc<<<nblk(g.nxy, BS), BS, 0, s>>>(g, ru, rv, rw));
}
void launch_init_faces(const Geo &g, const double *u, const double *v, const double *w, const double *rho,
                       double *ru, double *rv, double *rw, cudaStream_t s) {
    LAUNCH("init_faces", s, k_init_faces<<<nblk(g.nw, BS), BS, 0, s>>>(g, u, v, w, rho, ru, rv, rw));
    LAUNCH("wall_bc", s, k_wall_bc<<<nblk(g.nxy, BS), BS, 0, s>>>(g, ru, rv, rw));
}
void launch_wall_bc(const Geo &g, const double *ru, const double *rv, double *rw, cudaStream_t s) {
    LAUNCH("wall_bc", s, k_wall_bc<<<nblk(g.nxy, BS), BS, 0, s>>>(g, ru, rv, rw));
}
void launch_stage_begin(const Geo &g, CF5 sn, CF5 st, F5 x, double *pp, double *pi, double *th, double *Tp,
                        double *Om, cudaStream_t s, const double *rqv) {
    LAUNCH("stage_begin", s, k_stage_begin<<<nblk(g.nw, BS), BS, 0, s>>>(g, sn, st, x, pp, pi, th, Tp, Om, rqv));
}
void launch_slow_rhs(const Geo &g, const Phys &ph, CF5 st, double *pp, const double *th, Prep pr,
                     double *ux, double *vy, double *wz, double *mfx, double *mfy, double *rom, double *mu,
                     double *flux, F5 R, cudaStream_t s, const double *rtke, double *muh, double *tke_src,
                     const MoistIO *mio) {
    LAUNCH("prep", s, k_prep<<<nblk(g.nw, BS), BS, 0, s>>>(g, st, ux, vy, wz, mfx, mfy, rom));
    const int visc = (ph.closure == 1 || ph.closure == 2 || ph.closure == 4) ? 1 : 0;
    const int sgs = (visc || ph.surface == 1) ? 1 : 0;
    // advection, pressure gradient, buoyancy and Coriolis (the subgrid terms follow below)
    double *fx = flux, *fy = flux + g.nc, *fz = flux + 2 * g.nc;
    LAUNCH("flux_theta", s, k_flux_theta<<<nblk(g.nw, BS), BS, 0, s>>>(g, ph, pr, th, fx, fy, fz));
    LAUNCH("rhs_cells", s, k_rhs_cells<<<nblk(g.nc, BS), BS, 0, s>>>(g, ph, st, pr, fx, fy, fz, R.r, R.t));
    // momentum: fluxes of each component into the shared buffer, then its divergence
    const dim3 g3w((unsigned)((g.nx + 127) / 128), (unsigned)g.ny, (unsigned)(g.nz + 1));
    double *ax = flux, *ay = flux + g.nw, *az = flux + 2 * g.nw;
    if (ph.mom3) LAUNCH("flux_u", s, k_flux_u<1><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    else LAUNCH("flux_u", s, k_flux_u<0><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    LAUNCH("rhs_u", s, k_rhs_u<<<nblk(g.nc, BS), BS, 0, s>>>(g, ph, st, pp, ax, ay, az, R.u));
    if (ph.mom3) LAUNCH("flux_v", s, k_flux_v<1><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    else LAUNCH("flux_v", s, k_flux_v<0><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    LAUNCH("rhs_v", s, k_rhs_v<<<nblk(g.nc, BS), BS, 0, s>>>(g, ph, st, pp, ax, ay, az, R.v));
    if (ph.mom3) LAUNCH("flux_w", s, k_flux_w<1><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    else LAUNCH("flux_w", s, k_flux_w<0><<<g3w, 128, 0, s>>>(g, pr, ax, ay, az));
    LAUNCH("rhs_w", s, k_rhs_w<<<nblk(g.nw, BS), BS, 0, s>>>(g, ph, st, pp, ax, ay, az, R.w));
    if (sgs) {
        // subgrid stresses and heat fluxes, each edge and face once (the flux buffer is free again)
        Vel v{ux, vy, wz};
        double *e12 = flux, *e13 = flux + g.nw, *e23 = flux + 2 * g.nw;
        // the pressure and the mass fluxes are no longer needed in this stage's slow pass: they
        // take the diagonal stresses
        double *t11 = pp, *t22 = mfx, *t33 = mfy;
        Tke tk{rtke, th, muh, tke_src};
        if (visc) {
            LAUNCH("sgs_edges", s, k_sgs_edges<<<g3w, 128, 0, s>>>(g, v, e12, e13, e23));
            LAUNCH("sgs_mu", s, k_sgs_mu<<<nblk(g.nc, BS), BS, 0, s>>>(g, ph, v, st.r, e12, e13, e23, mu, t11, t22, t33,
                                                                       tk));
            if (ph.closure == 4)
                LAUNCH("tke_diff", s, k_tke_diff<<<nblk(g.nc, BS), BS, 0, s>>>(g, mu, rtke, st.r, tke_src));
        }
        LAUNCH("sgs_tau", s, k_sgs_tau<<<g3w, 128, 0, s>>>(g, ph, v, mu, st.r, th, visc, e12, e13, e23));
        const double *hk = ph.closure == 4 ? muh : mu;
        const double hs = ph.closure == 4 ? 1.0 : ph.rPr_t;
        LAUNCH("sgs_div", s, k_sgs_div<<<g3w, 128, 0, s>>>(g, ph, hk, hs, t11, t22, t33, st.r, th, visc, e12, e13, e23,
                                                           R));
        if (mio && ph.moist && visc)
            LAUNCH("moist_diff", s, k_moist_diff<<<nblk(g.nc, BS), BS, 0, s>>>(g, hk, hs, Q3{{ph.rqv, ph.rqc, ph.rqr}}, st.r,
                                                                           Q3w{{mio->src[0], mio->src[1], mio->src[2]}}));
    }
    if (mio && ph.moist && !(sgs && visc))
        for (int q = 0; q < 3; ++q) cudaMemsetAsync(mio->src[q], 0, g.nc * sizeof(double), s);
    if (mio && mio->ref[0]) {
        CF5 ref{mio->ref[0], mio->ref[1], mio->ref[2], mio->ref[3], mio->ref[4]};
        Q3 rq{{ph.rqv, ph.rqc, ph.rqr}}, rr{{mio->ref[5], mio->ref[6], mio->ref[7]}};
        Q3w qs{{mio->src[0], mio->src[1], mio->src[2]}};
        LAUNCH("relax", s, k_relax<<<nblk(g.nw, BS), BS, 0, s>>>(g, ph, st, ref, R, rq, rr, qs));
    }
}
void launch_tri_build(const Geo &g, const Phys &ph, const double *rho, const double *rt, const double *pi,
                      const double *th, double dtau, Tri tr, double *TX, double *TY, double *PX, double *PY,
                      double *THW, cudaStream_t s) {
    TriK tk;
    tk.E = dtau * ph.b2 * ph.b2;
    tk.EGg = tk.E * (dtau * 0.5 * ph.g);
    tk.cpg = dtau * (GAMMA * RD) * 0.5;
    tk.kgb = dtau * ph.g * (RD / CVD) * 0.5;
    tk.dpx = -tk.cpg;
    tk.hrdx = 0.5 * g.rdx;
    tk.hrdy = 0.5 * g.rdy;
    if (warp_columns(g))
        LAUNCH("tri_build", s, k_tri_build_warp<<<nblk(g.nxy, TRIW_WARPS), 32 * TRIW_WARPS, 0, s>>>(
                                   g, rho, rt, pi, th, tk, tr, TX, TY, PX, PY, THW, ph));
    else
        LAUNCH("tri_build", s, k_tri_build<<<nblk(g.nxy, col_block(g)), col_block(g), 0, s>>>(g, rho, rt, pi, th, tk, tr,
                                                                                          TX, TY, PX, PY, THW, ph));
}
void launch_substep(const Geo &g, const Phys &ph, Tri tr, const double *PX, const double *PY, const double *thw,
                    const double *TX, const double *TY, CF5 R, F5 x, double *Om, double *Tp, double *X0, double *Y0,
                    double *Ash,
                    double *msx, double *msy, double *msz, double dtau, cudaStream_t s) {
    const dim3 g3c((unsigned)((g.nx + 127) / 128), (unsigned)g.ny, (unsigned)g.nz);
    LAUNCH("sub_horiz", s, k_sub_horiz<<<nblk(g.nc, BS), BS, 0, s>>>(g, PX, PY, Tp, R.u, R.v, x.u, x.v, dtau));
    LAUNCH("sub_expl", s, k_sub_expl<<<g3c, 128, 0, s>>>(g, ph, thw, TX, TY, R.r, R.t, R.w, x, Om, Tp, X0, Y0, Ash,
                                                         msx, msy, msz, dtau));
    if (warp_columns(g))
        LAUNCH("sub_col", s, k_sub_col_warp<<<nblk(g.nxy, 4), 128, 0, s>>>(g.nz, g.nxy, tr.a, tr.cp, tr.im, tr.P, tr.Q,
                                                                           X0, Y0, x.w, Om, dtau * 0.5 * ph.g));
    else
    LAUNCH("sub_col", s, k_sub_col<<<nblk(g.nxy, col_block(g)), col_block(g), 0, s>>>(g.nz, g.nxy, tr.a, tr.cp, tr.im,
                                                                                      tr.P, tr.Q, X0, Y0, x.w, Om,
                                                                                      dtau * 0.5 * ph.g));
    LAUNCH("sub_fin", s, k_sub_fin<<<g3c, 128, 0, s>>>(g, ph, thw, Om, Ash, x, Tp, msz, dtau * ph.b2));
}
void launch_tracer_stage(const Geo &g, const Phys &ph, CF5 st, const double *rom, const double *snphi,
                         const double *msx, const double *msy, const double *msz, int nsub, double adt,
                         double *phi, double *flux, double *rphi, cudaStream_t s, const double *src, int clip) {
    const dim3 g3w((unsigned)((g.nx + 127) / 128), (unsigned)g.ny, (unsigned)(g.nz + 1));
    const dim3 g3c((unsigned)((g.nx + 127) / 128), (unsigned)g.ny, (unsigned)g.nz);
    double *fx = flux, *fy = flux + g.nw, *fz = flux + 2 * g.nw;
    LAUNCH("tracer_phi", s, k_tracer_phi<<<nblk(g.nc, BS), BS, 0, s>>>(g, rphi, st.r, phi));
    LAUNCH("tracer_flux", s, k_tracer_flux<<<g3w, 128, 0, s>>>(g, ph, st.u, st.v, rom, phi, msx, msy, msz,
                                                                1.0 / nsub, fx, fy, fz));
    LAUNCH(src ? "tke_update" : "tracer_update", s,
           k_tracer_update<<<g3c, 128, 0, s>>>(g, snphi, fx, fy, fz, src, clip, adt, rphi));
}
void launch_tracer_init(const Geo &g, const double *rho, const double *phi0, double *rphi, cudaStream_t s) {
    LAUNCH("tracer_init", s, k_tracer_init<<<nblk(g.nc, BS), BS, 0, s>>>(g, rho, phi0, rphi));
}
void launch_stage_end(const Geo &g, F5 st, CF5 x, cudaStream_t s) {
    LAUNCH("stage_end", s, k_stage_end<<<nblk(g.nw, BS), BS, 0, s>>>(g, st, x));
}
void launch_stage_nosub(const Geo &g, F5 st, CF5 sn, CF5 R, double adt, cudaStream_t s) {
    LAUNCH("stage_nosub", s, k_stage_nosub<<<nblk(g.nw, BS), BS, 0, s>>>(g, st, sn, R, adt));
}
void launch_diag(const Geo &g, CF5 st, double dt, double *part, double *out, cudaStream_t s) {
    LAUNCH("diag_partial", s, k_diag_partial<<<DIAG_BLOCKS, 256, 0, s>>>(g, st, part));
    LAUNCH("diag_final", s, k_diag_final<<<1, 32, 0, s>>>(part, DIAG_BLOCKS, dt, out));
}
void launch_diag_final(const double *part, int nparts, double dt, double *out, cudaStream_t s) {
    LAUNCH("diag_final", s, k_diag_final<<<1, 32, 0, s>>>(part, nparts, dt, out));
}
void launch_convert(const void *src, void *dst, long long n, int to_f64, cudaStream_t s) {
    if (to_f64)
        LAUNCH("f32_to_f64", s, k_f32_to_f64<<<nblk(n, BS), BS, 0, s>>>((const float *)src, (double *)dst, n));
    else
        LAUNCH("f64_to_f32", s, k_f64_to_f32<<<nblk(n, BS), BS, 0, s>>>((const double *)src, (float *)dst, n));
}

}  // namespace erfk
