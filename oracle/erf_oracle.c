/*
 * FP64 CPU oracle for one RK3 step of ERF's compressible dynamical core
 * (Lattanzi et al., "ERF: Energy Research and Forecasting Model", arXiv 2412.04395).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It
 * shares no code, header, table or helper with the CUDA library; the two meet only in the
 * seeded input generators (which hold none of the method's arithmetic).
 *
 * Plain loops in the order the paper states the method:
 *   Sec. 2.1  governing equations (Eqs. con, mom, theta), EOS, p' = p - p0, B = -(rho-rho0) g
 *   Sec. 3.1  low-storage RK3 (Wicker-Skamarock) with semi-implicit acoustic substeps,
 *             substep equations of App. C (beta_1, beta_2, beta_s = 0.1)
 *   Sec. 3.3  substep schedule (6 substeps per dt, 1 in the first stage, dt an even multiple)
 *   Sec. 3.4  Arakawa C-grid, terrain-following z = zeta + (1 - zeta/z_t)^beta h(x,y)
 *   App. A/B  Jacobian, contravariant Omega, discrete metric terms of Klemp (2003)
 *   Sec. 3.6  advection interpolants (upwind-5, centred-6, upwind-3, centred-4/2), WENO5
 *   Sec. 2.3  stress tensor tau = -2 mu (S - D); Smagorinsky-Lilly closure; a learned closure
 *             (Sec. 6, surrogate models) as cell-centre stresses from a model callback
 *   Sec. 3.8  HSE base state by Newton-Raphson; MOST bottom boundary
 * Readings where the paper is silent (constants, Smagorinsky form, WENO5 details, the
 * tridiagonal, divergence damping, wall ghost cells, MOST formulas) are stated beside the code
 * that takes them.
 *
 * Storage: C order [k][j][i], i fastest, periodic in x and y with every face stored once:
 *   cell (i,j,k) centred at ((i+1/2)dx, (j+1/2)dy);  x-face (i,j,k) at x = i dx (left face of cell i);
 *   y-face (i,j,k) at y = j dy;  w-face (i,j,k), k = 0..nz, bottom face of cell k;
 *   node (i,j,k) at (i dx, j dy, level k).
 * Built with -ffp-contract=off so no fused multiply-add changes the rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* physical constants: P00 is printed with the EOS (Sec. 2.1); R_d, c_p, kappa are not printed
 * (reading: the standard dry-air values used by WRF). g comes from the configuration. */
#define ORC_P00 1.0e5
#define ORC_RD 287.0
#define ORC_CP 1004.5
#define ORC_CV (ORC_CP - ORC_RD)
#define ORC_GAMMA (ORC_CP / ORC_CV)
#define ORC_KAPPA 0.4
/* moist air (Sec. 2.1, 2.4; not printed, readings): water-vapour gas constant, latent heat of
 * vaporisation, liquid-water density */
#define ORC_RV 461.5
#define ORC_LV 2.5e6
#define ORC_RHOW 1000.0

typedef struct {
    int32_t nx, ny, nz;
    double dx, dy;
    int32_t terrain_beta;     /* 1 = BTF, 3 = Sullivan (Sec. 3.4 canonical form) */
    double dt;
    int32_t n_substeps;       /* ns per dt (even); stage 1 uses 1 substep of dt/3 (Sec. 3.3) */
    int32_t substep_mode;     /* 0 = semi-implicit acoustic substeps, 1 = none (plain RK3) */
    int32_t acoustic_off;     /* test mode: drop every linear term of App. C, keep R^t */
    double beta_s, beta_d;    /* off-centering (App. C) and divergence damping (Sec. 3.1) */
    int32_t mom_adv;          /* interpolant order for momenta: 2,3,4,5,6 (Sec. 3.6) */
    int32_t scal_adv;         /* scalar scheme: 0 = WENO5-JS, 1 = WENO5-Z, 2..6 = linear interpolant */
    int32_t closure;          /* 0 none, 1 constant nu, 2 Smagorinsky, 3 learned (model callback) */
    double Cs, Pr_t, nu;
    double gravity;
    double f_cor, u_g, v_g;   /* f-plane Coriolis + geostrophic forcing (Sec. 3.7) */
    int32_t surface;          /* 0 slip wall, 1 MOST (constant z0, prescribed kinematic heat flux) */
    double z0, sfc_theta_flux;
    double theta_s, brunt_N, p_s;  /* base state: theta0 = theta_s exp(N^2 z/g) unless knots given */
    int32_t tracer;           /* 1: advance a passive scalar rho phi after the substeps (Sec. 3.1) */
    /* Rayleigh damping (Sec. 3.7, App. D): inverse timescale tau_max [1/s] at the domain top,
     * ramped by sin^2 from 0 at the bottom z_d of the damping layer; fields bitmask 1 = u, 2 = v,
     * 4 = w, 8 = theta (0 = off) */
    double ray_tau, ray_zd;
    int32_t ray_fields;
    /* moisture (Sec. 2.1 Eqs. nonprecip/precip, Sec. 2.4): 1 carries rho q_v, rho q_c, rho q_r with
     * the moist EOS and momentum terms, and applies Kessler microphysics after every RK3 step */
    int32_t moist;
    /* lateral relaxation zones (open x boundaries, Sec. 3.8 / Table D): every prognostic field
     * relaxes toward its initial value at rate relax_tau sin^2(pi/2 (1 - d/relax_width)) within
     * relax_width of an x-edge (d the distance to it); relax_tau = 0: off */
    double relax_tau, relax_width;
    /* anelastic equation set (Sec. 2.2): rho stays the base density rho0, the pressure
     * perturbation is the projection's (stored, not from the EOS) and the buoyancy is
     * rho0 g (theta - theta0) / theta0; the SSP-RK2 steps and the projection of Sec. 3.2 are
     * driven from oracle/anelastic.py */
    int32_t anelastic;
} orc_cfg;

typedef struct {
    orc_cfg c;
    int nx, ny, nz;
    size_t ncell, nw;          /* nx*ny*nz, nx*ny*(nz+1) */
    double zt;
    double *zeta;              /* nz+1 flat face heights */
    double *hnode;             /* ny*nx nodal terrain heights (zeros when flat) */
    int has_terrain;
    int n_knots;
    double *knot_z, *knot_th;
    /* geometry (App. B) */
    double *zn, *zw, *zc, *Hc, *Hx, *Hy, *hxi_x, *heta_y, *hxi_w, *heta_w;
    /* base state (Sec. 2, Sec. 3.8) */
    double *rho0, *th0, *p0;
    /* prognostic state */
    double *rho, *rt, *ru, *rv, *rw;
    int have_state;
    /* work arrays */
    double *sn[5];             /* S^n */
    double *pp, *pi, *th;      /* p', Exner, theta at stage t */
    double *R[5];              /* slow tendencies R_rho, R_Theta, R_U, R_V, R_W */
    double *X[5];              /* perturbations rho'', Theta'', U'', V'', W'' */
    double *Om;                /* Omega'' at w-faces (previous substep) */
    double *Tprev;             /* Theta'' of the previous substep (divergence damping) */
    double *fx, *fy, *fz, *mfx, *mfy, *rom, *ux, *vy, *wz, *mu;  /* slow-RHS scratch */
    /* passive scalar: rho phi, its S^n copy, and the sums over a stage's substeps of the
     * perturbation mass fluxes that advance rho'' (x-faces, y-faces, w-faces) */
    double *rphi, *sn_phi, *msx, *msy, *msz;
    /* Deardorff 1.5-order closure (closure 4): rho e (SGS kinetic energy per unit mass e), its S^n
     * copy, the stage's source rho (P + B - eps) + div(2 mu grad e) at cells, and the heat
     * diffusivity rho K_h at cells */
    double *rtke, *sn_tke, *tke_src, *muh;
    /* moisture: rho q_v, rho q_c, rho q_r (per unit dry mass), their S^n copies, the scalar
     * diffusion sources, the base-state vapour q_v0 at cells, and the accumulated surface
     * precipitation (metres of liquid water) per column */
    double *rq[3], *sn_q[3], *q_src[3], *qv0, *precip;
    /* relaxation zones: the reference (initial) state of every prognostic field */
    double *ref[5], *ref_q[3];
    /* anelastic pressure perturbation p' at cells */
    double *pa;
    /* learned closure (closure 3): a model evaluated on each stage state; it writes nine planes
     * of ncell values at cell centres, density-weighted: rho t11, rho t22, rho t33, rho t12,
     * rho t13, rho t23, rho h1, rho h2, rho h3 (kinematic stress [m^2/s^2] and SGS heat flux
     * [K m/s], the latter along +x, +y, +z) */
    void (*sgs_model)(void *user, const double *rho, const double *rt, const double *ru, const double *rv,
                      const double *rw, double *planes);
    void *sgs_user;
    double *sgs_planes;
} orc;

enum { F_RHO = 0, F_RT = 1, F_RU = 2, F_RV = 3, F_RW = 4 };

/* ------------------------------------------------------------------ index helpers */
static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static inline size_t IX(const orc *o, int i, int j, int k) {
    return ((size_t)k * o->ny + (size_t)wrap(j, o->ny)) * o->nx + (size_t)wrap(i, o->nx);
}
/* even reflection of a cell level about the walls (reading R4: three ghost layers) */
static inline int kref(int k, int nz) {
    while (k < 0 || k >= nz) {
        if (k < 0) k = -1 - k;
        if (k >= nz) k = 2 * nz - 1 - k;
    }
    return k;
}
/* cell-centred value with periodic x,y and even reflection in z */
static inline double CV(const orc *o, const double *f, int i, int j, int k) {
    return f[IX(o, i, j, kref(k, o->nz))];
}
/* w-face value (levels 0..nz) with odd reflection about the wall value: w(-m) = 2 w(0) - w(m) */
static double WV(const orc *o, const double *f, int i, int j, int k) {
    int nz = o->nz;
    if (k < 0) return 2.0 * f[IX(o, i, j, 0)] - WV(o, f, i, j, -k);
    if (k > nz) return 2.0 * f[IX(o, i, j, nz)] - WV(o, f, i, j, 2 * nz - k);
    return f[IX(o, i, j, k)];
}

/* ------------------------------------------------------------------ interpolants (Sec. 3.6) */
/* q[0..5] hold q_{m-3} .. q_{m+2}; the value returned is q at m-1/2.  s = sign of the
 * advecting normal momentum at m-1/2 (reading R2).  Centred 2nd/4th/6th and upwind 3rd/5th
 * exactly as printed. */
double orc_interp(const double *q, double s, int order) {
    double qm3 = q[0], qm2 = q[1], qm1 = q[2], qm = q[3], qp1 = q[4], qp2 = q[5];
    double c2 = 0.5 * (qm + qm1);
    double c4 = (7.0 / 12.0) * (qm + qm1) - (1.0 / 12.0) * (qp1 + qm2);
    double c6 = (37.0 / 60.0) * (qm + qm1) - (2.0 / 15.0) * (qp1 + qm2) + (1.0 / 60.0) * (qp2 + qm3);
    switch (order) {
    case 2: return c2;
    case 4: return c4;
    case 6: return c6;
    case 3: return c4 + (s / 12.0) * ((qp1 - qm2) - 3.0 * (qm - qm1));
    case 5: return c6 - (s / 60.0) * ((qp2 - qm3) - 5.0 * (qp1 - qm2) + 10.0 * (qm - qm1));
    default: return NAN;
    }
}

static inline double sgn(double x) { return (x > 0.0) ? 1.0 : ((x < 0.0) ? -1.0 : 0.0); }

/* WENO5 reconstruction at m-1/2 (Jiang & Shu 1996; WENO-Z of Borges et al. 2008 when zflag),
 * cited in Sec. 3.6.  Reading R7: candidate stencils, smoothness indicators with weights
 * 13/12 and 1/4, linear weights 1/10, 6/10, 3/10, eps = 1e-6, power 2 (JS) / tau5 = |b0-b2|,
 * power 1 (Z); upwind side chosen by the sign of the face momentum, >= 0 -> left. */
double orc_weno5(const double *q, double s, int zflag) {
    double vm2, vm1, v0, v1, v2;
    if (s >= 0.0) { vm2 = q[0]; vm1 = q[1]; v0 = q[2]; v1 = q[3]; v2 = q[4]; }
    else          { vm2 = q[5]; vm1 = q[4]; v0 = q[3]; v1 = q[2]; v2 = q[1]; }
    const double eps = 1.0e-6;
    double p0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
    double p1 = (-vm1 + 5.0 * v0 + 2.0 * v1) / 6.0;
    double p2 = (2.0 * v0 + 5.0 * v1 - v2) / 6.0;
    double b0 = (13.0 / 12.0) * (vm2 - 2.0 * vm1 + v0) * (vm2 - 2.0 * vm1 + v0)
              + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) * (vm2 - 4.0 * vm1 + 3.0 * v0);
    double b1 = (13.0 / 12.0) * (vm1 - 2.0 * v0 + v1) * (vm1 - 2.0 * v0 + v1)
              + 0.25 * (vm1 - v1) * (vm1 - v1);
    double b2 = (13.0 / 12.0) * (v0 - 2.0 * v1 + v2) * (v0 - 2.0 * v1 + v2)
              + 0.25 * (3.0 * v0 - 4.0 * v1 + v2) * (3.0 * v0 - 4.0 * v1 + v2);
    double a0, a1, a2;
    if (zflag) {
        double t5 = fabs(b0 - b2);
        a0 = 0.1 * (1.0 + t5 / (b0 + eps));
        a1 = 0.6 * (1.0 + t5 / (b1 + eps));
        a2 = 0.3 * (1.0 + t5 / (b2 + eps));
    } else {
        a0 = 0.1 / ((eps + b0) * (eps + b0));
        a1 = 0.6 / ((eps + b1) * (eps + b1));
        a2 = 0.3 / ((eps + b2) * (eps + b2));
    }
    double sa = a0 + a1 + a2;
    return (a0 * p0 + a1 * p1 + a2 * p2) / sa;
}

/* ------------------------------------------------------------------ EOS (Sec. 2.1) */
/* p = P00 (R_d rho theta / P00)^gamma (dry, q_v = 0); Exner pi = (p/P00)^(R_d/c_p). */
void orc_eos(double rt, double *p, double *pi) {
    double pr = ORC_P00 * pow(ORC_RD * rt / ORC_P00, ORC_GAMMA);
    *p = pr;
    *pi = pow(pr / ORC_P00, ORC_RD / ORC_CP);
}
/* EOS inverted for density at given pressure and potential temperature */
static double rho_of(double p, double theta) {
    return (ORC_P00 / (ORC_RD * theta)) * pow(p / ORC_P00, 1.0 / ORC_GAMMA);
}
/* the moist EOS of Sec. 2.1: p = P00 (R_d rho_d theta_d (1 + (R_v/R_d) q_v) / P00)^gamma
 * (rt = rho_d theta_d; q_v = 0 gives the dry EOS exactly) */
static void eos_q(double rt, double qv, double *p, double *pi) {
    orc_eos(rt * (1.0 + (ORC_RV / ORC_RD) * qv), p, pi);
}
/* total (moist) density rho_d (1 + q_v) of saturated-or-not air at pressure p, dry potential
 * temperature theta and vapour q_v (no condensate), from the moist EOS */
static double rho_m_of(double p, double theta, double qv) {
    return rho_of(p, theta * (1.0 + (ORC_RV / ORC_RD) * qv)) * (1.0 + qv);
}

/* ------------------------------------------------------------------ tridiagonal (Thomas) */
/* rows r = 0..n-1: a[r] x[r-1] + b[r] x[r] + c[r] x[r+1] = d[r]  (a[0], c[n-1] ignored) */
void orc_thomas(int n, const double *a, const double *b, const double *c, const double *d, double *x) {
    double *cp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (n > 0) {
        cp[0] = c[0] / b[0];
        dp[0] = d[0] / b[0];
        for (int r = 1; r < n; ++r) {
            double m = b[r] - a[r] * cp[r - 1];
            cp[r] = c[r] / m;
            dp[r] = (d[r] - a[r] * dp[r - 1]) / m;
        }
        x[n - 1] = dp[n - 1];
        for (int r = n - 2; r >= 0; --r) x[r] = dp[r] - cp[r] * x[r + 1];
    }
    free(cp);
    free(dp);
}

/* ------------------------------------------------------------------ base-state profile */
static double theta0_at(const orc *o, double z) {
    if (o->n_knots > 0) {           /* piecewise-linear sounding, constant beyond the ends */
        if (z <= o->knot_z[0]) return o->knot_th[0];
        for (int n = 1; n < o->n_knots; ++n)
            if (z <= o->knot_z[n]) {
                double t = (z - o->knot_z[n - 1]) / (o->knot_z[n] - o->knot_z[n - 1]);
                return o->knot_th[n - 1] + t * (o->knot_th[n] - o->knot_th[n - 1]);
            }
        return o->knot_th[o->n_knots - 1];
    }
    double g = o->c.gravity;
    if (o->c.brunt_N == 0.0 || g == 0.0) return o->c.theta_s;
    return o->c.theta_s * exp(o->c.brunt_N * o->c.brunt_N * z / g);
}

/* base-state water vapour q_v0(z): piecewise-linear sounding, constant beyond the ends (0 without one) */
static double qv0_at(int n, const double *kz, const double *kq, double z) {
    if (n <= 0) return 0.0;
    if (z <= kz[0]) return kq[0];
    for (int m = 1; m < n; ++m)
        if (z <= kz[m]) {
            double t = (z - kz[m - 1]) / (kz[m] - kz[m - 1]);
            return kq[m - 1] + t * (kq[m] - kq[m - 1]);
        }
    return kq[n - 1];
}

/* HSE column by Newton-Raphson (Sec. 3.8): from p_s at z = 0, trapezoidal hydrostatic steps
 *   p_k = p_{k-1} - g (z_k - z_{k-1}) (rho_{k-1} + rho_k)/2,  rho_k = EOS^-1(p_k, theta0(z_k)),
 * solved for p_k; z are the column's cell-centre heights.  p0 is then re-evaluated from the
 * EOS of rho0 theta0 so that an undisturbed state has p' = 0 exactly. */
/* The same column with moisture (Sec. 3.8: the moist background state matches the input
 * profiles of theta and q_v at every height): the hydrostatic density is the total density
 * rho_d (1 + q_v0) from the moist EOS; qcol = NULL is the dry column. */
static void hse_column_q(int nz, const double *zcol, const double *thcol, const double *qcol, double p_s,
                         double th_surf, double q_surf, double g, double *rho0, double *p0out) {
    double p_prev = p_s, rho_prev = rho_m_of(p_s, th_surf, q_surf), z_prev = 0.0;
    for (int k = 0; k < nz; ++k) {
        double dz = zcol[k] - z_prev, th = thcol[k], q = qcol ? qcol[k] : 0.0;
        double p = p_prev - g * dz * rho_prev;
        for (int it = 0; it < 50; ++it) {
            double r = rho_m_of(p, th, q);
            double f = p - p_prev + 0.5 * g * dz * (rho_prev + r);
            double df = 1.0 + 0.5 * g * dz * r / (ORC_GAMMA * p);
            double dp = -f / df;
            p += dp;
            if (fabs(dp) <= 1.0e-14 * fabs(p)) break;
        }
        double r = rho_m_of(p, th, q);
        rho0[k] = r;
        p0out[k] = p;
        p_prev = p; rho_prev = r; z_prev = zcol[k];
    }
}
void orc_hse_column(int nz, const double *zcol, const double *thcol, double p_s, double th_surf,
                    double g, double *rho0, double *p0out) {
    hse_column_q(nz, zcol, thcol, NULL, p_s, th_surf, 0.0, g, rho0, p0out);
}

/* ------------------------------------------------------------------ setup */
static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

void orc_destroy(orc *o);

orc *orc_create2(const orc_cfg *cfg, const double *zeta, const double *hnode, int n_knots, const double *knot_z,
                 const double *knot_th, int n_qknots, const double *qknot_z, const double *qknot_v);
orc *orc_create(const orc_cfg *cfg, const double *zeta, const double *hnode,
                int n_knots, const double *knot_z, const double *knot_th) {
    return orc_create2(cfg, zeta, hnode, n_knots, knot_z, knot_th, 0, NULL, NULL);
}
/* with a base-state water-vapour sounding (moist configurations) */
orc *orc_create2(const orc_cfg *cfg, const double *zeta, const double *hnode, int n_knots, const double *knot_z,
                 const double *knot_th, int n_qknots, const double *qknot_z, const double *qknot_v) {
    orc *o = (orc *)calloc(1, sizeof(orc));
    o->c = *cfg;
    int nx = o->nx = cfg->nx, ny = o->ny = cfg->ny, nz = o->nz = cfg->nz;
    o->ncell = (size_t)nx * ny * nz;
    o->nw = (size_t)nx * ny * (nz + 1);
    o->zeta = dalloc(nz + 1);
    memcpy(o->zeta, zeta, sizeof(double) * (nz + 1));
    o->zt = zeta[nz];
    o->hnode = dalloc((size_t)nx * ny);
    o->has_terrain = 0;
    if (hnode) {
        memcpy(o->hnode, hnode, sizeof(double) * (size_t)nx * ny);
        for (size_t n = 0; n < (size_t)nx * ny; ++n) if (hnode[n] != 0.0) o->has_terrain = 1;
    }
    o->n_knots = n_knots;
    if (n_knots > 0) {
        o->knot_z = dalloc(n_knots); o->knot_th = dalloc(n_knots);
        memcpy(o->knot_z, knot_z, sizeof(double) * n_knots);
        memcpy(o->knot_th, knot_th, sizeof(double) * n_knots);
    }
    size_t NC = o->ncell, NW = o->nw;
    o->zn = dalloc(NW); o->zw = dalloc(NW); o->zc = dalloc(NC); o->Hc = dalloc(NC);
    o->Hx = dalloc(NC); o->Hy = dalloc(NC); o->hxi_x = dalloc(NC); o->heta_y = dalloc(NC);
    o->hxi_w = dalloc(NW); o->heta_w = dalloc(NW);
    o->rho0 = dalloc(NC); o->th0 = dalloc(NC); o->p0 = dalloc(NC);
    o->rho = dalloc(NC); o->rt = dalloc(NC); o->ru = dalloc(NC); o->rv = dalloc(NC); o->rw = dalloc(NW);
    for (int f = 0; f < 5; ++f) {
        size_t n = (f == F_RW) ? NW : NC;
        o->sn[f] = dalloc(n); o->R[f] = dalloc(n); o->X[f] = dalloc(n);
    }
    o->pp = dalloc(NC); o->pi = dalloc(NC); o->th = dalloc(NC);
    o->Om = dalloc(NW); o->Tprev = dalloc(NC);
    o->fx = dalloc(NW); o->fy = dalloc(NW); o->fz = dalloc(NW);
    o->mfx = dalloc(NC); o->mfy = dalloc(NC); o->rom = dalloc(NW);
    o->ux = dalloc(NC); o->vy = dalloc(NC); o->wz = dalloc(NW); o->mu = dalloc(NC);
    o->rphi = dalloc(NC); o->sn_phi = dalloc(NC); o->msx = dalloc(NC); o->msy = dalloc(NC); o->msz = dalloc(NW);
    o->rtke = dalloc(NC); o->sn_tke = dalloc(NC); o->tke_src = dalloc(NC); o->muh = dalloc(NC);
    for (int q = 0; q < 3; ++q) {
        o->rq[q] = dalloc(NC); o->sn_q[q] = dalloc(NC); o->q_src[q] = dalloc(NC); o->ref_q[q] = dalloc(NC);
    }
    for (int f = 0; f < 5; ++f) o->ref[f] = dalloc(f == F_RW ? NW : NC);
    o->qv0 = dalloc(NC); o->precip = dalloc((size_t)nx * ny);
    o->pa = dalloc(NC);

    /* node heights, App. B + canonical smoothing z = zeta + (1 - zeta/z_t)^beta h (Sec. 3.4) */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = pow(1.0 - o->zeta[k] / o->zt, (double)cfg->terrain_beta);
                o->zn[IX(o, i, j, k)] = o->zeta[k] + s * o->hnode[(size_t)j * nx + i];
            }
    /* w-face centre heights: 4 surrounding nodes; cell centre: average of the two w-faces (= 8 nodes) */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                o->zw[IX(o, i, j, k)] = 0.25 * (o->zn[IX(o, i, j, k)] + o->zn[IX(o, i + 1, j, k)]
                                              + o->zn[IX(o, i, j + 1, k)] + o->zn[IX(o, i + 1, j + 1, k)]);
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                o->zc[c] = 0.5 * (o->zw[IX(o, i, j, k)] + o->zw[IX(o, i, j, k + 1)]);
                o->Hc[c] = o->zw[IX(o, i, j, k + 1)] - o->zw[IX(o, i, j, k)];
                o->Hx[c] = 0.5 * ((o->zn[IX(o, i, j, k + 1)] - o->zn[IX(o, i, j, k)])
                                + (o->zn[IX(o, i, j + 1, k + 1)] - o->zn[IX(o, i, j + 1, k)]));
                o->Hy[c] = 0.5 * ((o->zn[IX(o, i, j, k + 1)] - o->zn[IX(o, i, j, k)])
                                + (o->zn[IX(o, i + 1, j, k + 1)] - o->zn[IX(o, i + 1, j, k)]));
            }
    /* h_xi at x-faces from cell-centre heights (App. B, pressure gradient); h_eta likewise */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                o->hxi_x[IX(o, i, j, k)] = (o->zc[IX(o, i, j, k)] - o->zc[IX(o, i - 1, j, k)]) / cfg->dx;
                o->heta_y[IX(o, i, j, k)] = (o->zc[IX(o, i, j, k)] - o->zc[IX(o, i, j - 1, k)]) / cfg->dy;
            }
    /* 4th-order h_xi, h_eta at w-faces from 4-node-averaged face heights (App. B, Omega) */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                o->hxi_w[IX(o, i, j, k)] = (o->zw[IX(o, i - 2, j, k)] - o->zw[IX(o, i + 2, j, k)]
                    + 8.0 * (o->zw[IX(o, i + 1, j, k)] - o->zw[IX(o, i - 1, j, k)])) / (12.0 * cfg->dx);
                o->heta_w[IX(o, i, j, k)] = (o->zw[IX(o, i, j - 2, k)] - o->zw[IX(o, i, j + 2, k)]
                    + 8.0 * (o->zw[IX(o, i, j + 1, k)] - o->zw[IX(o, i, j - 1, k)])) / (12.0 * cfg->dy);
            }
    /* base state per column (HSE in physical height, Sec. 2 and Sec. 3.8) */
    double *zcol = dalloc(nz), *thcol = dalloc(nz), *rcol = dalloc(nz), *pcol = dalloc(nz), *qcol = dalloc(nz);
    int moist = cfg->moist && n_qknots > 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            for (int k = 0; k < nz; ++k) {
                zcol[k] = o->zc[IX(o, i, j, k)];
                thcol[k] = theta0_at(o, zcol[k]);
                qcol[k] = moist ? qv0_at(n_qknots, qknot_z, qknot_v, zcol[k]) : 0.0;
            }
            if (moist)
                hse_column_q(nz, zcol, thcol, qcol, cfg->p_s, theta0_at(o, 0.0),
                             qv0_at(n_qknots, qknot_z, qknot_v, 0.0), cfg->gravity, rcol, pcol);
            else
                orc_hse_column(nz, zcol, thcol, cfg->p_s, theta0_at(o, 0.0), cfg->gravity, rcol, pcol);
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k);
                double pr, pie;
                o->rho0[c] = rcol[k];                     /* total density (moist base states) */
                o->th0[c] = thcol[k];
                o->qv0[c] = qcol[k];
                /* p0 from the EOS of the base dry density rho0 / (1 + q_v0), so that p' = 0 exactly */
                eos_q(rcol[k] / (1.0 + qcol[k]) * thcol[k], qcol[k], &pr, &pie);
                o->p0[c] = pr;
            }
        }
    free(zcol); free(thcol); free(rcol); free(pcol); free(qcol);
    return o;
}

void orc_destroy(orc *o) {
    if (!o) return;
    double **ptrs[] = {&o->zeta, &o->hnode, &o->knot_z, &o->knot_th, &o->zn, &o->zw, &o->zc, &o->Hc,
                       &o->Hx, &o->Hy, &o->hxi_x, &o->heta_y, &o->hxi_w, &o->heta_w, &o->rho0,
                       &o->th0, &o->p0, &o->rho, &o->rt, &o->ru, &o->rv, &o->rw, &o->pp, &o->pi,
                       &o->th, &o->Om, &o->Tprev, &o->fx, &o->fy, &o->fz, &o->mfx, &o->mfy,
                       &o->rom, &o->ux, &o->vy, &o->wz, &o->mu, &o->rphi, &o->sn_phi, &o->msx,
                       &o->msy, &o->msz, &o->sgs_planes, &o->rtke, &o->sn_tke, &o->tke_src, &o->muh};
    for (size_t n = 0; n < sizeof(ptrs) / sizeof(ptrs[0]); ++n) free(*ptrs[n]);
    for (int f = 0; f < 5; ++f) { free(o->sn[f]); free(o->R[f]); free(o->X[f]); free(o->ref[f]); }
    for (int q = 0; q < 3; ++q) { free(o->rq[q]); free(o->sn_q[q]); free(o->q_src[q]); free(o->ref_q[q]); }
    free(o->qv0); free(o->precip); free(o->pa);
    free(o);
}

/* ------------------------------------------------------------------ boundary: Omega = 0 at walls */
/* rho*Omega = rho w - h_xi <rho u> - h_eta <rho v> at w-faces with the 4-point averages of App. B;
 * levels outside the domain are even reflections (reading R4). */
static double avg4_u(const orc *o, const double *fu, int i, int j, int k) {
    return 0.25 * (CV(o, fu, i, j, k - 1) + CV(o, fu, i + 1, j, k - 1) + CV(o, fu, i, j, k) + CV(o, fu, i + 1, j, k));
}
static double avg4_v(const orc *o, const double *fv, int i, int j, int k) {
    return 0.25 * (CV(o, fv, i, j, k - 1) + CV(o, fv, i, j + 1, k - 1) + CV(o, fv, i, j, k) + CV(o, fv, i, j + 1, k));
}
/* h_xi <U> + h_eta <V> at w-face (i,j,k): the part of W that is not contravariant */
static double metric_shift(const orc *o, const double *fu, const double *fv, int i, int j, int k) {
    if (!o->has_terrain) return 0.0;
    size_t w = IX(o, i, j, k);
    return o->hxi_w[w] * avg4_u(o, fu, i, j, k) + o->heta_w[w] * avg4_v(o, fv, i, j, k);
}
static void apply_wall_bc(orc *o, double *rw, const double *ru, const double *rv) {
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i) {
            rw[IX(o, i, j, 0)] = metric_shift(o, ru, rv, i, j, 0);
            rw[IX(o, i, j, o->nz)] = 0.0;
        }
}

/* ------------------------------------------------------------------ stage EOS pass */
static void eos_pass(orc *o, const double *rho, const double *rt) {
    const int moist = o->c.moist;
    if (o->c.anelastic) {   /* Sec. 2.2: p' from the projection, no EOS; pi is not used */
        for (size_t c = 0; c < o->ncell; ++c) {
            o->pp[c] = o->pa[c];
            o->pi[c] = 1.0;
            o->th[c] = rt[c] / rho[c];
        }
        return;
    }
#pragma omp parallel for
    for (long c = 0; c < (long)o->ncell; ++c) {
        double p, pie;
        if (moist) eos_q(rt[c], o->rq[0][c] / rho[c], &p, &pie);   /* q_v of the stage state */
        else orc_eos(rt[c], &p, &pie);
        o->pp[c] = p - o->p0[c];
        o->pi[c] = pie;
        o->th[c] = rt[c] / rho[c];
    }
}

/* ------------------------------------------------------------------ MOST (reading R15) */
/* Businger-Dyer (Dyer 1974) momentum stability function; zeta = z/L */
static double psi_m(double zeta) {
    if (zeta < 0.0) {
        double x = pow(1.0 - 16.0 * zeta, 0.25);
        return 2.0 * log(0.5 * (1.0 + x)) + log(0.5 * (1.0 + x * x)) - 2.0 * atan(x) + 0.5 * M_PI;
    }
    return -5.0 * zeta;
}
double orc_psi_m(double zeta) { return psi_m(zeta); }

/* friction velocity for wind speed U at height z1 over roughness z0 with kinematic heat flux Q:
 * neutral start, then 5 fixed-point iterations through the Obukhov length, z1/L in [-5, 1]. */
double orc_ustar(double U, double z1, double z0, double Q, double theta, double g) {
    double lz = log(z1 / z0);
    double us = ORC_KAPPA * U / lz;
    if (Q == 0.0 || g == 0.0) return us;
    for (int it = 0; it < 5; ++it) {
        double zeta;
        if (us <= 0.0) zeta = (Q > 0.0) ? -5.0 : 1.0;
        else {
            double L = -us * us * us * theta / (ORC_KAPPA * g * Q);
            zeta = z1 / L;
        }
        if (zeta < -5.0) zeta = -5.0;
        if (zeta > 1.0) zeta = 1.0;
        us = ORC_KAPPA * U / (lz - psi_m(zeta));
    }
    return us;
}

/* ------------------------------------------------------------------ slow right-hand side R^t */
/* Eq. con, Eq. mom, Eq. theta evaluated at the stage state (Sec. 3.1: "source term f(S)").
 * Flux form in terrain-following coordinates (App. A, Eq. terraindiv): divergences are formed
 * with face heights H (= h_zeta dzeta at that face) and rho*Omega on w-faces, and divided by
 * the height of the control volume. */
static void slow_rhs(orc *o, const double *rho, const double *rt, const double *ru,
                     const double *rv, const double *rw) {
    const orc_cfg *C = &o->c;
    int nx = o->nx, ny = o->ny, nz = o->nz;
    double dx = C->dx, dy = C->dy, g = C->gravity;
    double *Rr = o->R[F_RHO], *Rt = o->R[F_RT], *Ru = o->R[F_RU], *Rv = o->R[F_RV], *Rw = o->R[F_RW];
    memset(Rw, 0, sizeof(double) * o->nw);

    eos_pass(o, rho, rt);
    if (C->moist)
        for (int q = 0; q < 3; ++q) memset(o->q_src[q], 0, sizeof(double) * o->ncell);
    /* moisture (Eq. mom): pressure gradient and buoyancy scaled by 1 / (1 + q_v + q_c), buoyancy of the
     * total density rho_m = rho_d (1 + q_v + q_c + q_r); qvc = q_v + q_c, qt = rho_m - rho_d at cells */
    double *qvc = NULL, *qtm = NULL;
    if (C->moist) {
        qvc = dalloc(o->ncell); qtm = dalloc(o->ncell);
        for (size_t c = 0; c < o->ncell; ++c) {
            qvc[c] = (o->rq[0][c] + o->rq[1][c]) / rho[c];
            qtm[c] = o->rq[0][c] + o->rq[1][c] + o->rq[2][c];
        }
    }
    /* mass fluxes per unit length (Sec. 3.6: normal momentum at the face) and rho*Omega */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                o->mfx[c] = o->Hx[c] * ru[c];
                o->mfy[c] = o->Hy[c] * rv[c];
                /* primitive velocities at faces: u = rho u / rho averaged to the face */
                o->ux[c] = ru[c] / (0.5 * (CV(o, rho, i - 1, j, k) + rho[c]));
                o->vy[c] = rv[c] / (0.5 * (CV(o, rho, i, j - 1, k) + rho[c]));
            }
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t w = IX(o, i, j, k);
                o->rom[w] = (k == 0 || k == nz) ? 0.0 : rw[w] - metric_shift(o, ru, rv, i, j, k);
                double rb = 0.5 * (CV(o, rho, i, j, k - 1) + CV(o, rho, i, j, k));
                o->wz[w] = rw[w] / rb;
            }

    /* --- continuity, Eq. con */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double div = (o->mfx[IX(o, i + 1, j, k)] - o->mfx[c]) / dx
                           + (o->mfy[IX(o, i, j + 1, k)] - o->mfy[c]) / dy
                           + (o->rom[IX(o, i, j, k + 1)] - o->rom[IX(o, i, j, k)]);
                Rr[c] = -div / o->Hc[c];
            }

    /* --- potential temperature advection, Eq. theta: face flux = normal momentum x WENO5(theta) */
    int zf = (C->scal_adv == 1);
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double q[6];
                size_t w = IX(o, i, j, k);
                if (k < nz) {
                    size_t c = w;
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->th, i - 3 + m, j, k);
                    o->fx[c] = o->mfx[c] * (C->scal_adv <= 1 ? orc_weno5(q, sgn(o->mfx[c]), zf)
                                                              : orc_interp(q, sgn(o->mfx[c]), C->scal_adv));
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->th, i, j - 3 + m, k);
                    o->fy[c] = o->mfy[c] * (C->scal_adv <= 1 ? orc_weno5(q, sgn(o->mfy[c]), zf)
                                                              : orc_interp(q, sgn(o->mfy[c]), C->scal_adv));
                }
                if (k == 0 || k == nz) { o->fz[w] = 0.0; continue; }   /* walls: no advective flux */
                for (int m = 0; m < 6; ++m) q[m] = CV(o, o->th, i, j, k - 3 + m);
                o->fz[w] = o->rom[w] * (C->scal_adv <= 1 ? orc_weno5(q, sgn(o->rom[w]), zf)
                                                          : orc_interp(q, sgn(o->rom[w]), C->scal_adv));
            }
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double div = (o->fx[IX(o, i + 1, j, k)] - o->fx[c]) / dx
                           + (o->fy[IX(o, i, j + 1, k)] - o->fy[c]) / dy
                           + (o->fz[IX(o, i, j, k + 1)] - o->fz[IX(o, i, j, k)]);
                Rt[c] = -div / o->Hc[c];
            }

    /* --- momentum advection, Eq. mom: advecting momentum spatially averaged to the flux
     * location (reading R5), primitive velocity interpolated with the order mom_adv. */
    int ord = C->mom_adv;
    /* x-momentum: x-fluxes at cell centres, y-fluxes at xy-edges, z-fluxes at xz-edges */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double q[6];
                size_t w = IX(o, i, j, k);
                if (k < nz) {
                    size_t c = w;
                    double adv = 0.5 * (o->mfx[c] + o->mfx[IX(o, i + 1, j, k)]);      /* at centre (i,j,k) */
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->ux, i - 2 + m, j, k);
                    o->fx[c] = adv * orc_interp(q, sgn(adv), ord);
                    adv = 0.5 * (o->mfy[IX(o, i - 1, j, k)] + o->mfy[c]);              /* at edge (x-face i, y-face j) */
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->ux, i, j - 3 + m, k);
                    o->fy[c] = adv * orc_interp(q, sgn(adv), ord);
                }
                if (k == 0 || k == nz) { o->fz[w] = 0.0; continue; }
                double adv = 0.5 * (o->rom[IX(o, i - 1, j, k)] + o->rom[w]);           /* at edge (x-face i, w-face k) */
                for (int m = 0; m < 6; ++m) q[m] = CV(o, o->ux, i, j, k - 3 + m);
                o->fz[w] = adv * orc_interp(q, sgn(adv), ord);
            }
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double div = (o->fx[c] - o->fx[IX(o, i - 1, j, k)]) / dx
                           + (o->fy[IX(o, i, j + 1, k)] - o->fy[c]) / dy
                           + (o->fz[IX(o, i, j, k + 1)] - o->fz[IX(o, i, j, k)]);
                Ru[c] = -div / o->Hx[c];
            }
    /* y-momentum */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double q[6];
                size_t w = IX(o, i, j, k);
                if (k < nz) {
                    size_t c = w;
                    double adv = 0.5 * (o->mfx[IX(o, i, j - 1, k)] + o->mfx[c]);      /* at edge (x-face i, y-face j) */
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->vy, i - 3 + m, j, k);
                    o->fx[c] = adv * orc_interp(q, sgn(adv), ord);
                    adv = 0.5 * (o->mfy[c] + o->mfy[IX(o, i, j + 1, k)]);              /* at centre (i,j,k) */
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, o->vy, i, j - 2 + m, k);
                    o->fy[c] = adv * orc_interp(q, sgn(adv), ord);
                }
                if (k == 0 || k == nz) { o->fz[w] = 0.0; continue; }
                double adv = 0.5 * (o->rom[IX(o, i, j - 1, k)] + o->rom[w]);           /* at edge (y-face j, w-face k) */
                for (int m = 0; m < 6; ++m) q[m] = CV(o, o->vy, i, j, k - 3 + m);
                o->fz[w] = adv * orc_interp(q, sgn(adv), ord);
            }
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double div = (o->fx[IX(o, i + 1, j, k)] - o->fx[c]) / dx
                           + (o->fy[c] - o->fy[IX(o, i, j - 1, k)]) / dy
                           + (o->fz[IX(o, i, j, k + 1)] - o->fz[IX(o, i, j, k)]);
                Rv[c] = -div / o->Hy[c];
            }
    /* z-momentum at interior w-faces k = 1..nz-1: x/y fluxes at edges, z fluxes at cell centres */
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double q[6];
                size_t w = IX(o, i, j, k);
                if (k >= 1 && k < nz) {
                    double adv = 0.5 * (o->mfx[IX(o, i, j, k - 1)] + o->mfx[IX(o, i, j, k)]);   /* edge (x-face i, w-face k) */
                    for (int m = 0; m < 6; ++m) q[m] = WV(o, o->wz, i - 3 + m, j, k);
                    o->fx[w] = adv * orc_interp(q, sgn(adv), ord);
                    adv = 0.5 * (o->mfy[IX(o, i, j, k - 1)] + o->mfy[IX(o, i, j, k)]);          /* edge (y-face j, w-face k) */
                    for (int m = 0; m < 6; ++m) q[m] = WV(o, o->wz, i, j - 3 + m, k);
                    o->fy[w] = adv * orc_interp(q, sgn(adv), ord);
                }
                if (k < nz) {   /* at cell centre (i,j,k), between w-faces k and k+1 */
                    double adv = 0.5 * (o->rom[w] + o->rom[IX(o, i, j, k + 1)]);
                    for (int m = 0; m < 6; ++m) q[m] = WV(o, o->wz, i, j, k - 2 + m);
                    o->fz[w] = adv * orc_interp(q, sgn(adv), ord);
                }
            }
    #pragma omp parallel for
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t w = IX(o, i, j, k);
                double Hw = o->zc[IX(o, i, j, k)] - o->zc[IX(o, i, j, k - 1)];
                double div = (o->fx[IX(o, i + 1, j, k)] - o->fx[w]) / dx
                           + (o->fy[IX(o, i, j + 1, k)] - o->fy[w]) / dy
                           + (o->fz[IX(o, i, j, k)] - o->fz[IX(o, i, j, k - 1)]);
                Rw[w] = -div / Hw;
            }

    /* --- pressure gradient (App. B terrain form) and buoyancy (Sec. 2.1, reading R3) */
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double px = (o->pp[c] - o->pp[IX(o, i - 1, j, k)]) / dx;
                double py = (o->pp[c] - o->pp[IX(o, i, j - 1, k)]) / dy;
                if (o->has_terrain && nz > 1) {
                    /* (p_zeta/h_zeta) centred over cell-centre heights, one-sided at the walls */
                    double d[4];
                    int ii[4] = {i, i - 1, i, i}, jj[4] = {j, j, j, j - 1};
                    for (int n = 0; n < 4; ++n) {
                        int kl = (k == 0) ? 0 : k - 1, ku = (k == nz - 1) ? nz - 1 : k + 1;
                        d[n] = (o->pp[IX(o, ii[n], jj[n], ku)] - o->pp[IX(o, ii[n], jj[n], kl)])
                             / (o->zc[IX(o, ii[n], jj[n], ku)] - o->zc[IX(o, ii[n], jj[n], kl)]);
                    }
                    px -= 0.5 * o->hxi_x[c] * (d[0] + d[1]);
                    py -= 0.5 * o->heta_y[c] * (d[2] + d[3]);
                }
                if (qvc) {
                    px /= 1.0 + 0.5 * (qvc[IX(o, i - 1, j, k)] + qvc[c]);
                    py /= 1.0 + 0.5 * (qvc[IX(o, i, j - 1, k)] + qvc[c]);
                }
                Ru[c] -= px;
                Rv[c] -= py;
            }
    #pragma omp parallel for
    for (int k = 1; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t w = IX(o, i, j, k), c = IX(o, i, j, k), cm = IX(o, i, j, k - 1);
                double pz = (o->pp[c] - o->pp[cm]) / (o->zc[c] - o->zc[cm]);
                if (C->anelastic) {
                    /* Sec. 2.2: B = rho0 g (theta - theta0) / theta0, the face mean of the two cells */
                    double Bm = o->rho0[cm] * g * (o->th[cm] - o->th0[cm]) / o->th0[cm];
                    double Bc = o->rho0[c] * g * (o->th[c] - o->th0[c]) / o->th0[c];
                    Rw[w] += -pz + 0.5 * (Bm + Bc);
                } else if (qtm) {
                    double B = 0.5 * (-g * (rho[cm] + qtm[cm] - o->rho0[cm]) - g * (rho[c] + qtm[c] - o->rho0[c]));
                    Rw[w] += (-pz + B) / (1.0 + 0.5 * (qvc[cm] + qvc[c]));
                } else {
                    double B = 0.5 * (-g * (rho[cm] - o->rho0[cm]) - g * (rho[c] - o->rho0[c]));
                    Rw[w] += -pz + B;
                }
            }

    /* --- Coriolis and geostrophic forcing on an f-plane (Sec. 3.7) */
    if (C->f_cor != 0.0)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, k);
                    double rvx = 0.25 * (CV(o, rv, i - 1, j, k) + rv[c] + CV(o, rv, i - 1, j + 1, k) + CV(o, rv, i, j + 1, k));
                    double rux = 0.25 * (CV(o, ru, i, j - 1, k) + CV(o, ru, i + 1, j - 1, k) + ru[c] + CV(o, ru, i + 1, j, k));
                    double rhx = 0.5 * (CV(o, rho, i - 1, j, k) + rho[c]);
                    double rhy = 0.5 * (CV(o, rho, i, j - 1, k) + rho[c]);
                    Ru[c] += C->f_cor * (rvx - rhx * C->v_g);
                    Rv[c] -= C->f_cor * (rux - rhy * C->u_g);
                }

    /* --- subgrid stress and heat flux: -div(tau), div(rho alpha grad theta) (Eq. stresstensor;
     * reading R6 for the Smagorinsky-Lilly form on a flat, possibly stretched grid) */
    if (C->closure >= 1 || C->surface == 1) {
        /* strain at cell centres (diagonal) and edges (off-diagonal), velocities at faces */
        double *S11 = dalloc(o->ncell), *S22 = dalloc(o->ncell), *S33 = dalloc(o->ncell);
        double *S12 = dalloc(o->ncell), *S13 = dalloc(o->nw), *S23 = dalloc(o->nw);
        double *t11 = dalloc(o->ncell), *t22 = dalloc(o->ncell), *t33 = dalloc(o->ncell);
        double *t12 = dalloc(o->ncell), *t13 = dalloc(o->nw), *t23 = dalloc(o->nw);
        double *hx = dalloc(o->ncell), *hy = dalloc(o->ncell), *hz = dalloc(o->nw);
        int visc = (C->closure == 1 || C->closure == 2 || C->closure == 4);
        #pragma omp parallel for
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, k);
                    S11[c] = (o->ux[IX(o, i + 1, j, k)] - o->ux[c]) / dx;
                    S22[c] = (o->vy[IX(o, i, j + 1, k)] - o->vy[c]) / dy;
                    S33[c] = (o->wz[IX(o, i, j, k + 1)] - o->wz[IX(o, i, j, k)]) / o->Hc[c];
                    S12[c] = 0.5 * ((o->ux[c] - o->ux[IX(o, i, j - 1, k)]) / dy + (o->vy[c] - o->vy[IX(o, i - 1, j, k)]) / dx);
                }
        #pragma omp parallel for
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t w = IX(o, i, j, k);
                    if (k == 0 || k == nz) { S13[w] = 0.0; S23[w] = 0.0; continue; }   /* slip walls */
                    double dzc = o->zc[IX(o, i, j, k)] - o->zc[IX(o, i, j, k - 1)];
                    S13[w] = 0.5 * ((o->ux[IX(o, i, j, k)] - o->ux[IX(o, i, j, k - 1)]) / dzc
                                  + (o->wz[w] - o->wz[IX(o, i - 1, j, k)]) / dx);
                    S23[w] = 0.5 * ((o->vy[IX(o, i, j, k)] - o->vy[IX(o, i, j, k - 1)]) / dzc
                                  + (o->wz[w] - o->wz[IX(o, i, j - 1, k)]) / dy);
                }
        /* eddy viscosity mu = rho (Cs Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij), edges averaged to centres */
        #pragma omp parallel for
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, k);
                    double s12 = 0.25 * (S12[c] + S12[IX(o, i + 1, j, k)] + S12[IX(o, i, j + 1, k)] + S12[IX(o, i + 1, j + 1, k)]);
                    double s13 = 0.25 * (S13[IX(o, i, j, k)] + S13[IX(o, i + 1, j, k)] + S13[IX(o, i, j, k + 1)] + S13[IX(o, i + 1, j, k + 1)]);
                    double s23 = 0.25 * (S23[IX(o, i, j, k)] + S23[IX(o, i, j + 1, k)] + S23[IX(o, i, j, k + 1)] + S23[IX(o, i, j + 1, k + 1)]);
                    double SS = S11[c] * S11[c] + S22[c] * S22[c] + S33[c] * S33[c]
                              + 2.0 * (s12 * s12 + s13 * s13 + s23 * s23);
                    double mu = 0.0;
                    if (C->closure == 2) {
                        double Delta = cbrt(dx * dy * o->Hc[c]);
                        mu = rho[c] * (C->Cs * Delta) * (C->Cs * Delta) * sqrt(2.0 * SS);
                    } else if (C->closure == 1) {
                        mu = rho[c] * C->nu;
                    }
                    double dv = S11[c] + S22[c] + S33[c];
                    if (C->closure == 4) {
                        /* Deardorff (1980) 1.5-order closure with the coefficients of Moeng (1984):
                         * mixing length l = Delta, or 0.76 sqrt(e)/N in stable stratification when
                         * shorter; K_m = 0.1 l sqrt(e); K_h = (1 + 2 l/Delta) K_m; dissipation
                         * C_eps e^(3/2)/l with C_eps = 0.19 + 0.51 l/Delta.  N^2 = (g/theta) dtheta/dz
                         * from the cells above and below (one-sided at the walls).  The shear
                         * production is the energy the resolved flow loses to the stress
                         * tau = -2 mu (S - D): -tau_ij S_ij / rho = 2 K_m (S_ij S_ij - (S_kk)^2/3). */
                        double e = o->rtke[c] / rho[c];
                        if (e < 0.0) e = 0.0;
                        double Delta = cbrt(dx * dy * o->Hc[c]);
                        int kl = (k == 0) ? 0 : k - 1, ku = (k == nz - 1) ? nz - 1 : k + 1;
                        double N2 = 0.0;
                        if (ku > kl) {
                            size_t cl = IX(o, i, j, kl), cu = IX(o, i, j, ku);
                            N2 = g / o->th[c] * (o->th[cu] - o->th[cl]) / (o->zc[cu] - o->zc[cl]);
                        }
                        double l = Delta;
                        if (N2 > 0.0 && e > 0.0) {
                            double ls = 0.76 * sqrt(e) / sqrt(N2);
                            if (ls < l) l = ls;
                        }
                        double Km = 0.1 * l * sqrt(e);
                        double Kh = (1.0 + 2.0 * l / Delta) * Km;
                        mu = rho[c] * Km;
                        o->muh[c] = rho[c] * Kh;
                        double P = 2.0 * Km * (SS - dv * dv / 3.0);
                        double B = -Kh * N2;
                        double eps = (0.19 + 0.51 * l / Delta) * e * sqrt(e) / l;
                        o->tke_src[c] = rho[c] * (P + B - eps);
                    }
                    o->mu[c] = mu;
                    t11[c] = -2.0 * mu * (S11[c] - dv / 3.0);
                    t22[c] = -2.0 * mu * (S22[c] - dv / 3.0);
                    t33[c] = -2.0 * mu * (S33[c] - dv / 3.0);
                }
        #pragma omp parallel for
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t w = IX(o, i, j, k);
                    if (k < nz) {
                        size_t c = w;
                        double me = 0.25 * (o->mu[IX(o, i - 1, j - 1, k)] + o->mu[IX(o, i, j - 1, k)]
                                          + o->mu[IX(o, i - 1, j, k)] + o->mu[c]);
                        t12[c] = -2.0 * me * S12[c];
                        /* heat diffusivity rho alpha_theta: mu / Pr_t, or rho K_h (Deardorff) */
                        double ax = (C->closure == 4) ? 0.5 * (o->muh[IX(o, i - 1, j, k)] + o->muh[c])
                                                      : 0.5 * (o->mu[IX(o, i - 1, j, k)] + o->mu[c]) / C->Pr_t;
                        double ay = (C->closure == 4) ? 0.5 * (o->muh[IX(o, i, j - 1, k)] + o->muh[c])
                                                      : 0.5 * (o->mu[IX(o, i, j - 1, k)] + o->mu[c]) / C->Pr_t;
                        hx[c] = ax * (o->th[c] - o->th[IX(o, i - 1, j, k)]) / dx;
                        hy[c] = ay * (o->th[c] - o->th[IX(o, i, j - 1, k)]) / dy;
                    }
                    if (k == 0 || k == nz) { t13[w] = 0.0; t23[w] = 0.0; hz[w] = 0.0; continue; }
                    double mxz = 0.25 * (o->mu[IX(o, i - 1, j, k - 1)] + o->mu[IX(o, i, j, k - 1)]
                                       + o->mu[IX(o, i - 1, j, k)] + o->mu[IX(o, i, j, k)]);
                    double myz = 0.25 * (o->mu[IX(o, i, j - 1, k - 1)] + o->mu[IX(o, i, j, k - 1)]
                                       + o->mu[IX(o, i, j - 1, k)] + o->mu[IX(o, i, j, k)]);
                    t13[w] = -2.0 * mxz * S13[w];
                    t23[w] = -2.0 * myz * S23[w];
                    double dzc = o->zc[IX(o, i, j, k)] - o->zc[IX(o, i, j, k - 1)];
                    double az = (C->closure == 4) ? 0.5 * (o->muh[IX(o, i, j, k - 1)] + o->muh[IX(o, i, j, k)])
                                                  : 0.5 * (o->mu[IX(o, i, j, k - 1)] + o->mu[IX(o, i, j, k)]) / C->Pr_t;
                    hz[w] = az * (o->th[IX(o, i, j, k)] - o->th[IX(o, i, j, k - 1)]) / dzc;
                }
        if (!visc) {   /* MOST without a closure: only the surface fluxes below */
            memset(t11, 0, sizeof(double) * o->ncell); memset(t22, 0, sizeof(double) * o->ncell);
            memset(t33, 0, sizeof(double) * o->ncell); memset(t12, 0, sizeof(double) * o->ncell);
            memset(t13, 0, sizeof(double) * o->nw); memset(t23, 0, sizeof(double) * o->nw);
            memset(hx, 0, sizeof(double) * o->ncell); memset(hy, 0, sizeof(double) * o->ncell);
            memset(hz, 0, sizeof(double) * o->nw);
        }
        if (C->closure == 3) {
            /* learned closure: the model's cell-centre stresses t11, t22, t33 enter as they are;
             * t12, t13, t23 are carried to their edges by the mean of the four cells around each
             * edge (zero at the lid; the ground edges take MOST below, else zero); the heat flux
             * goes to each face as the mean of its two cells, with the sign of the down-gradient
             * flux h above (h = -rho h_model) */
            o->sgs_model(o->sgs_user, rho, rt, ru, rv, rw, o->sgs_planes);
            const double *P = o->sgs_planes;
            size_t N = o->ncell;
            #pragma omp parallel for
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t c = IX(o, i, j, k);
                        t11[c] = P[c];
                        t22[c] = P[N + c];
                        t33[c] = P[2 * N + c];
                        t12[c] = 0.25 * (P[3 * N + IX(o, i - 1, j - 1, k)] + P[3 * N + IX(o, i, j - 1, k)]
                                       + P[3 * N + IX(o, i - 1, j, k)] + P[3 * N + c]);
                        hx[c] = -0.5 * (P[6 * N + IX(o, i - 1, j, k)] + P[6 * N + c]);
                        hy[c] = -0.5 * (P[7 * N + IX(o, i, j - 1, k)] + P[7 * N + c]);
                        if (k == 0) continue;
                        t13[c] = 0.25 * (P[4 * N + IX(o, i - 1, j, k - 1)] + P[4 * N + IX(o, i, j, k - 1)]
                                       + P[4 * N + IX(o, i - 1, j, k)] + P[4 * N + c]);
                        t23[c] = 0.25 * (P[5 * N + IX(o, i, j - 1, k - 1)] + P[5 * N + IX(o, i, j, k - 1)]
                                       + P[5 * N + IX(o, i, j - 1, k)] + P[5 * N + c]);
                        hz[c] = -0.5 * (P[8 * N + IX(o, i, j, k - 1)] + P[8 * N + c]);
                    }
        }
        if (C->surface == 1) {
            /* MOST surface stress tau_i3 = -rho u*^2 u_i/|U| at the bottom edges; upward heat flux rho Q */
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, 0);
                    double z1 = o->zc[c] - o->zw[c];
                    double u = o->ux[c];
                    double v = 0.25 * (o->vy[IX(o, i - 1, j, 0)] + o->vy[c] + o->vy[IX(o, i - 1, j + 1, 0)] + o->vy[IX(o, i, j + 1, 0)]);
                    double U = sqrt(u * u + v * v);
                    double thf = 0.5 * (o->th[IX(o, i - 1, j, 0)] + o->th[c]);
                    double rhf = 0.5 * (rho[IX(o, i - 1, j, 0)] + rho[c]);
                    if (U > 0.0) {
                        double us = orc_ustar(U, z1, C->z0, C->sfc_theta_flux, thf, g);
                        t13[c] = -rhf * us * us * u / U;
                    }
                    u = 0.25 * (o->ux[IX(o, i, j - 1, 0)] + o->ux[IX(o, i + 1, j - 1, 0)] + o->ux[c] + o->ux[IX(o, i + 1, j, 0)]);
                    v = o->vy[c];
                    U = sqrt(u * u + v * v);
                    thf = 0.5 * (o->th[IX(o, i, j - 1, 0)] + o->th[c]);
                    rhf = 0.5 * (rho[IX(o, i, j - 1, 0)] + rho[c]);
                    if (U > 0.0) {
                        double us = orc_ustar(U, z1, C->z0, C->sfc_theta_flux, thf, g);
                        t23[c] = -rhf * us * us * v / U;
                    }
                    /* upward kinematic flux Q into the domain: rho alpha dtheta/dz = -rho Q at the surface */
                    hz[c] = -rho[c] * C->sfc_theta_flux;
                }
        }
        #pragma omp parallel for
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, k);
                    double H = o->Hc[c];
                    Ru[c] -= (t11[c] - t11[IX(o, i - 1, j, k)]) / dx + (t12[IX(o, i, j + 1, k)] - t12[c]) / dy
                           + (t13[IX(o, i, j, k + 1)] - t13[IX(o, i, j, k)]) / H;
                    Rv[c] -= (t12[IX(o, i + 1, j, k)] - t12[c]) / dx + (t22[c] - t22[IX(o, i, j - 1, k)]) / dy
                           + (t23[IX(o, i, j, k + 1)] - t23[IX(o, i, j, k)]) / H;
                    Rt[c] += (hx[IX(o, i + 1, j, k)] - hx[c]) / dx + (hy[IX(o, i, j + 1, k)] - hy[c]) / dy
                           + (hz[IX(o, i, j, k + 1)] - hz[IX(o, i, j, k)]) / H;
                }
        #pragma omp parallel for
        for (int k = 1; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t w = IX(o, i, j, k);
                    double dzc = o->zc[IX(o, i, j, k)] - o->zc[IX(o, i, j, k - 1)];
                    Rw[w] -= (t13[IX(o, i + 1, j, k)] - t13[w]) / dx + (t23[IX(o, i, j + 1, k)] - t23[w]) / dy
                           + (t33[IX(o, i, j, k)] - t33[IX(o, i, j, k - 1)]) / dzc;
                }
        if (C->moist) {
            /* moisture diffusion (Eq. nonprecip, precip): div(rho alpha_q grad q) with alpha_q the
             * heat diffusivity of the closure (mu / Pr_t, or rho K_h), no flux through the walls */
            for (int q = 0; q < 3; ++q) {
                double *qq = dalloc(o->ncell);
                for (size_t c = 0; c < o->ncell; ++c) qq[c] = o->rq[q][c] / rho[c];
                #pragma omp parallel for
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j)
                        for (int i = 0; i < nx; ++i) {
                            size_t c = IX(o, i, j, k);
                            if (!visc) { o->q_src[q][c] = 0.0; continue; }
                            const double *hk = (C->closure == 4) ? o->muh : o->mu;
                            double hs = (C->closure == 4) ? 1.0 : 1.0 / C->Pr_t;
                            size_t cxm = IX(o, i - 1, j, k), cxp = IX(o, i + 1, j, k);
                            size_t cym = IX(o, i, j - 1, k), cyp = IX(o, i, j + 1, k);
                            double fxm = 0.5 * (hk[cxm] + hk[c]) * hs * (qq[c] - qq[cxm]) / dx;
                            double fxp = 0.5 * (hk[c] + hk[cxp]) * hs * (qq[cxp] - qq[c]) / dx;
                            double fym = 0.5 * (hk[cym] + hk[c]) * hs * (qq[c] - qq[cym]) / dy;
                            double fyp = 0.5 * (hk[c] + hk[cyp]) * hs * (qq[cyp] - qq[c]) / dy;
                            double fzm = 0.0, fzp = 0.0;
                            if (k > 0) {
                                size_t cm = IX(o, i, j, k - 1);
                                fzm = 0.5 * (hk[cm] + hk[c]) * hs * (qq[c] - qq[cm]) / (o->zc[c] - o->zc[cm]);
                            }
                            if (k < nz - 1) {
                                size_t cp = IX(o, i, j, k + 1);
                                fzp = 0.5 * (hk[c] + hk[cp]) * hs * (qq[cp] - qq[c]) / (o->zc[cp] - o->zc[c]);
                            }
                            o->q_src[q][c] = (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / o->Hc[c];
                        }
                free(qq);
            }
        }
        if (C->closure == 4) {
            /* transport of e by the SGS eddies: div(rho 2 K_m grad e), face coefficient the mean
             * of the two cells' 2 mu; no flux through the walls */
            double *e = dalloc(o->ncell);
            for (size_t c = 0; c < o->ncell; ++c) { double v = o->rtke[c] / rho[c]; e[c] = v > 0.0 ? v : 0.0; }
            #pragma omp parallel for
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t c = IX(o, i, j, k);
                        size_t cxm = IX(o, i - 1, j, k), cxp = IX(o, i + 1, j, k);
                        size_t cym = IX(o, i, j - 1, k), cyp = IX(o, i, j + 1, k);
                        double fxm = (o->mu[cxm] + o->mu[c]) * (e[c] - e[cxm]) / dx;
                        double fxp = (o->mu[c] + o->mu[cxp]) * (e[cxp] - e[c]) / dx;
                        double fym = (o->mu[cym] + o->mu[c]) * (e[c] - e[cym]) / dy;
                        double fyp = (o->mu[c] + o->mu[cyp]) * (e[cyp] - e[c]) / dy;
                        double fzm = 0.0, fzp = 0.0;
                        if (k > 0) {
                            size_t cm = IX(o, i, j, k - 1);
                            fzm = (o->mu[cm] + o->mu[c]) * (e[c] - e[cm]) / (o->zc[c] - o->zc[cm]);
                        }
                        if (k < nz - 1) {
                            size_t cp = IX(o, i, j, k + 1);
                            fzp = (o->mu[c] + o->mu[cp]) * (e[cp] - e[c]) / (o->zc[cp] - o->zc[c]);
                        }
                        o->tke_src[c] += (fxp - fxm) / dx + (fyp - fym) / dy + (fzp - fzm) / o->Hc[c];
                    }
            free(e);
        }
        free(S11); free(S22); free(S33); free(S12); free(S13); free(S23);
        free(t11); free(t22); free(t33); free(t12); free(t13); free(t23);
        free(hx); free(hy); free(hz);
    }

    /* --- Rayleigh damping (Sec. 3.7; App. D: strength an inverse timescale, sin^2 ramp from 0 at
     * the bottom z_d of the layer to tau_max at the top z_t).  Reading: each damped quantity relaxes
     * toward its reference at its own physical height - u, v toward the geostrophic wind (u_g,
     * v_g), w toward 0, theta toward the base state theta0 - as -tau(z) rho (phi - phi_ref) in the
     * tendency of rho phi (the face density the mean of the two cells). */
    if (C->ray_tau > 0.0 && C->ray_fields != 0) {
        const double zd = C->ray_zd, zt = o->zt;
        #pragma omp parallel for
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IX(o, i, j, k), cxm = IX(o, i - 1, j, k), cym = IX(o, i, j - 1, k);
                    double z, t;
                    if (C->ray_fields & 8) {
                        z = o->zc[c];
                        t = (z > zd) ? C->ray_tau * pow(sin(0.5 * M_PI * (z - zd) / (zt - zd)), 2.0) : 0.0;
                        Rt[c] -= t * (rt[c] - rho[c] * o->th0[c]);
                    }
                    if (C->ray_fields & 1) {
                        z = 0.5 * (o->zc[cxm] + o->zc[c]);
                        t = (z > zd) ? C->ray_tau * pow(sin(0.5 * M_PI * (z - zd) / (zt - zd)), 2.0) : 0.0;
                        Ru[c] -= t * (ru[c] - 0.5 * (rho[cxm] + rho[c]) * C->u_g);
                    }
                    if (C->ray_fields & 2) {
                        z = 0.5 * (o->zc[cym] + o->zc[c]);
                        t = (z > zd) ? C->ray_tau * pow(sin(0.5 * M_PI * (z - zd) / (zt - zd)), 2.0) : 0.0;
                        Rv[c] -= t * (rv[c] - 0.5 * (rho[cym] + rho[c]) * C->v_g);
                    }
                    if ((C->ray_fields & 4) && k >= 1) {
                        size_t w = IX(o, i, j, k);
                        z = o->zw[w];
                        t = (z > zd) ? C->ray_tau * pow(sin(0.5 * M_PI * (z - zd) / (zt - zd)), 2.0) : 0.0;
                        Rw[w] -= t * rw[w];
                    }
                }
    }

    /* --- lateral relaxation zones (open x boundaries; Sec. 3.8 nudging toward boundary data, here
     * the initial state): -tau_r(d) (S - S_ref), tau_r = relax_tau sin^2(pi/2 (1 - d/W)) for d < W,
     * d the distance of the point from the nearer x-edge (cells at x_c, x-faces at x = i dx) */
    if (C->relax_tau > 0.0 && C->relax_width > 0.0) {
        const double Lx = nx * dx, W = C->relax_width;
        #pragma omp parallel for
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double xc = (i + 0.5) * dx, xf = i * dx;
                    double dc = xc < Lx - xc ? xc : Lx - xc, df = xf < Lx - xf ? xf : Lx - xf;
                    double tc = dc < W ? C->relax_tau * pow(sin(0.5 * M_PI * (1.0 - dc / W)), 2.0) : 0.0;
                    double tf = df < W ? C->relax_tau * pow(sin(0.5 * M_PI * (1.0 - df / W)), 2.0) : 0.0;
                    size_t c = IX(o, i, j, k);
                    if (k < nz) {
                        Rr[c] -= tc * (rho[c] - o->ref[F_RHO][c]);
                        Rt[c] -= tc * (rt[c] - o->ref[F_RT][c]);
                        Ru[c] -= tf * (ru[c] - o->ref[F_RU][c]);
                        Rv[c] -= tc * (rv[c] - o->ref[F_RV][c]);
                        if (C->moist)
                            for (int q = 0; q < 3; ++q) o->q_src[q][c] -= tc * (o->rq[q][c] - o->ref_q[q][c]);
                    }
                    if (k >= 1 && k < nz) Rw[c] -= tc * (rw[c] - o->ref[F_RW][c]);
                }
    }
    free(qvc); free(qtm);
}

/* stage-t mixing ratios q_v + q_c and q_v + q_c + q_r at a cell */
static inline double qvc_at(const orc *o, const double *rho_t, size_t c) {
    return (o->rq[0][c] + o->rq[1][c]) / rho_t[c];
}
static inline double qt_at(const orc *o, const double *rho_t, size_t c) {
    return (o->rq[0][c] + o->rq[1][c] + o->rq[2][c]) / rho_t[c];
}

/* ------------------------------------------------------------------ acoustic substep (App. C) */
/* One substep of length dtau on the perturbations X'' about the stage state (rho^t, Theta^t,
 * pi^t, theta^t held fixed).  Horizontal momenta forward (divergence-damped pressure term,
 * reading R10), then per column the W'', Theta'', rho'' rows reduced to one tridiagonal
 * system in Omega'' (reading R11), solved by the Thomas algorithm, and back-substituted. */
static void substep(orc *o, const double *rho_t, const double *rt_t, double dtau) {
    const orc_cfg *C = &o->c;
    int nx = o->nx, ny = o->ny, nz = o->nz;
    double dx = C->dx, dy = C->dy, g = C->gravity;
    double b1 = 0.5 * (1.0 - C->beta_s), b2 = 0.5 * (1.0 + C->beta_s);
    double lin = C->acoustic_off ? 0.0 : 1.0;     /* switch for every linear (acoustic) term */
    double *Xr = o->X[F_RHO], *Xt = o->X[F_RT], *Xu = o->X[F_RU], *Xv = o->X[F_RV], *Xw = o->X[F_RW];
    double *Rr = o->R[F_RHO], *Rt = o->R[F_RT], *Ru = o->R[F_RU], *Rv = o->R[F_RV], *Rw = o->R[F_RW];
    double gRd = ORC_GAMMA * ORC_RD;

    /* Theta~ = Theta''^tau + beta_d (Theta''^tau - Theta''^{tau - dtau}) */
    double *Tt = dalloc(o->ncell);
    for (size_t c = 0; c < o->ncell; ++c) Tt[c] = Xt[c] + C->beta_d * (Xt[c] - o->Tprev[c]);

    /* horizontal momenta: Delta U'' = dtau(-gamma R_d pi^t (dTheta~/dxi - h_xi/h_zeta dTheta~/dzeta) + R_U) */
    double *Un = dalloc(o->ncell), *Vn = dalloc(o->ncell);
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double gx = (Tt[c] - Tt[IX(o, i - 1, j, k)]) / dx;
                double gy = (Tt[c] - Tt[IX(o, i, j - 1, k)]) / dy;
                if (o->has_terrain && nz > 1) {
                    double d[4];
                    int ii[4] = {i, i - 1, i, i}, jj[4] = {j, j, j, j - 1};
                    for (int n = 0; n < 4; ++n) {
                        int kl = (k == 0) ? 0 : k - 1, ku = (k == nz - 1) ? nz - 1 : k + 1;
                        d[n] = (Tt[IX(o, ii[n], jj[n], ku)] - Tt[IX(o, ii[n], jj[n], kl)])
                             / (o->zc[IX(o, ii[n], jj[n], ku)] - o->zc[IX(o, ii[n], jj[n], kl)]);
                    }
                    gx -= 0.5 * o->hxi_x[c] * (d[0] + d[1]);
                    gy -= 0.5 * o->heta_y[c] * (d[2] + d[3]);
                }
                double pix = 0.5 * (o->pi[IX(o, i - 1, j, k)] + o->pi[c]);
                double piy = 0.5 * (o->pi[IX(o, i, j - 1, k)] + o->pi[c]);
                if (C->moist) {   /* App. C: gamma R_d pi^t / (1 + q_v^t + q_c^t) at the face */
                    pix /= 1.0 + 0.5 * (qvc_at(o, rho_t, IX(o, i - 1, j, k)) + qvc_at(o, rho_t, c));
                    piy /= 1.0 + 0.5 * (qvc_at(o, rho_t, IX(o, i, j - 1, k)) + qvc_at(o, rho_t, c));
                }
                Un[c] = Xu[c] + dtau * (-lin * gRd * pix * gx + Ru[c]);
                Vn[c] = Xv[c] + dtau * (-lin * gRd * piy * gy + Rv[c]);
            }
    memcpy(o->Tprev, Xt, sizeof(double) * o->ncell);
    memcpy(Xu, Un, sizeof(double) * o->ncell);
    memcpy(Xv, Vn, sizeof(double) * o->ncell);
    /* the horizontal perturbation mass fluxes that advance rho'' in this substep */
    for (size_t c = 0; c < o->ncell; ++c) {
        o->msx[c] += lin * o->Hx[c] * Un[c];
        o->msy[c] += lin * o->Hy[c] * Vn[c];
    }
    free(Un); free(Vn); free(Tt);

    /* per column: vertical implicit solve */
#pragma omp parallel
    {
    double *Ts = dalloc(nz), *Rs = dalloc(nz), *thw = dalloc(nz + 1), *A = dalloc(nz + 1);
    double *a = dalloc(nz), *b = dalloc(nz), *cc = dalloc(nz), *d = dalloc(nz), *x = dalloc(nz);
    double *Om = dalloc(nz + 1);
#pragma omp for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            /* theta^t at w-faces (walls take the adjacent cell) */
            for (int k = 0; k <= nz; ++k)
                thw[k] = 0.5 * (CV(o, o->th, i, j, k - 1) + CV(o, o->th, i, j, k));
            for (int k = 0; k <= nz; ++k) A[k] = (k == nz) ? 0.0 : metric_shift(o, Xu, Xv, i, j, k);
            /* explicit parts Theta*, rho*: horizontal divergence of the new U'', V'' and the
             * beta_1 part of the vertical flux of the old Omega'' */
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k), cxp = IX(o, i + 1, j, k), cyp = IX(o, i, j + 1, k);
                double thxm = 0.5 * (o->th[IX(o, i - 1, j, k)] + o->th[c]);
                double thxp = 0.5 * (o->th[c] + o->th[cxp]);
                double thym = 0.5 * (o->th[IX(o, i, j - 1, k)] + o->th[c]);
                double thyp = 0.5 * (o->th[c] + o->th[cyp]);
                double divM = (o->Hx[cxp] * Xu[cxp] - o->Hx[c] * Xu[c]) / dx
                            + (o->Hy[cyp] * Xv[cyp] - o->Hy[c] * Xv[c]) / dy;
                double divT = (o->Hx[cxp] * Xu[cxp] * thxp - o->Hx[c] * Xu[c] * thxm) / dx
                            + (o->Hy[cyp] * Xv[cyp] * thyp - o->Hy[c] * Xv[c] * thym) / dy;
                double wo_p = o->Om[IX(o, i, j, k + 1)], wo_m = o->Om[IX(o, i, j, k)];
                double H = o->Hc[c];
                Ts[k] = Xt[c] + dtau * (-lin * divT / H - lin * b1 * (wo_p * thw[k + 1] - wo_m * thw[k]) / H + Rt[c]);
                Rs[k] = Xr[c] + dtau * (-lin * divM / H - lin * b1 * (wo_p - wo_m) / H + Rr[c]);
            }
            /* tridiagonal rows for Omega''_k, k = 1..nz-1 (Omega'' = 0 on the walls) */
            double E = lin * dtau * b2 * b2, Gg = lin * dtau * 0.5 * g;
            for (int k = 1; k < nz; ++k) {
                size_t c = IX(o, i, j, k), cm = IX(o, i, j, k - 1), w = IX(o, i, j, k);
                double dzc = o->zc[c] - o->zc[cm];
                double pib = 0.5 * (o->pi[cm] + o->pi[c]);
                double rhob = 0.5 * (rho_t[cm] + rho_t[c]);
                double Cpg = gRd * pib / dzc;                                  /* gamma R_d pi / (h_zeta dzeta) */
                double Cbp = g * rhob * (ORC_RD / ORC_CV) * 0.5 * o->pi[c] / (rt_t[c] * pib);   /* reading R13 */
                double Cbm = g * rhob * (ORC_RD / ORC_CV) * 0.5 * o->pi[cm] / (rt_t[cm] * pib);
                if (C->moist) {
                    /* App. C: the pressure term over 1 + q_v + q_c, the Theta'' buoyancy times
                     * rho_d / rho_m = 1 / (1 + q_v + q_c + q_r), all face means of stage-t cells */
                    Cpg /= 1.0 + 0.5 * (qvc_at(o, rho_t, cm) + qvc_at(o, rho_t, c));
                    double rm = 1.0 + 0.5 * (qt_at(o, rho_t, cm) + qt_at(o, rho_t, c));
                    Cbp /= rm;
                    Cbm /= rm;
                }
                double P = lin * dtau * (-Cpg + Cbp), Q = lin * dtau * (Cpg + Cbm);
                double Hk = o->Hc[c], Hm = o->Hc[cm];
                double X0k = b1 * Xt[c] + b2 * Ts[k], X0m = b1 * Xt[cm] + b2 * Ts[k - 1];
                double Y0k = b1 * Xr[c] + b2 * Rs[k], Y0m = b1 * Xr[cm] + b2 * Rs[k - 1];
                int r = k - 1;
                a[r] = E * (Gg - Q * thw[k - 1]) / Hm;
                b[r] = 1.0 - P * E * thw[k] / Hk + Q * E * thw[k] / Hm + Gg * E * (1.0 / Hk - 1.0 / Hm);
                cc[r] = E * (P * thw[k + 1] - Gg) / Hk;
                d[r] = Xw[w] - A[k] + dtau * Rw[w] + P * X0k + Q * X0m - Gg * (Y0k + Y0m);
            }
            if (nz > 1) orc_thomas(nz - 1, a, b, cc, d, x);
            Om[0] = 0.0; Om[nz] = 0.0;
            for (int k = 1; k < nz; ++k) Om[k] = x[k - 1];
            for (int k = 0; k <= nz; ++k) {
                size_t w = IX(o, i, j, k);
                /* vertical perturbation mass flux of the rho'' update: beta_1 old + beta_2 new */
                o->msz[w] += lin * (b1 * o->Om[w] + b2 * Om[k]);
                Xw[w] = Om[k] + A[k];
                o->Om[w] = Om[k];
            }
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k);
                double H = o->Hc[c];
                Xt[c] = Ts[k] - lin * dtau * b2 * (Om[k + 1] * thw[k + 1] - Om[k] * thw[k]) / H;
                Xr[c] = Rs[k] - lin * dtau * b2 * (Om[k + 1] - Om[k]) / H;
            }
        }
    free(Ts); free(Rs); free(thw); free(A); free(a); free(b); free(cc); free(d); free(x); free(Om);
    }
}

/* ------------------------------------------------------------------ passive scalar (Sec. 3.1) */
/* Scalars do not take part in the substeps: after them, rho phi advances over the stage as
 * without substepping, rho phi^(s) = rho phi^n + alpha_s dt R_phi(phi^t), except that the normal
 * momenta of the advective fluxes are the average over the stage's substeps of those that
 * advanced rho (stage momentum + perturbation flux of each substep).  With that average,
 * rho phi / rho stays 1 for phi = 1 (rho^(s) = rho^n - alpha_s dt div <M>).  phi^t is
 * interpolated like theta (WENO5 or the linear interpolant of scal_adv). */
/* The same stage update serves every transported scalar q (rho phi, and rho e of the Deardorff
 * closure): rho q^(s) = rho q^n + alpha_s dt (-div F(q^t) / H + src), src the scalar's own source
 * at the stage state (NULL: none); clip = 1 keeps rho q >= 0 (the SGS energy). */
static void scalar_stage(orc *o, double *rq, const double *sn_q, const double *src, int clip,
                         const double *rho_t, double adt, int nsub) {
    const orc_cfg *C = &o->c;
    int nx = o->nx, ny = o->ny, nz = o->nz;
    double dx = C->dx, dy = C->dy;
    int zf = (C->scal_adv == 1);
    double *phi = dalloc(o->ncell), *F[3] = {dalloc(o->ncell), dalloc(o->ncell), dalloc(o->nw)};
    for (size_t c = 0; c < o->ncell; ++c) phi[c] = rq[c] / rho_t[c];
    #pragma omp parallel for
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double q[6];
                size_t w = IX(o, i, j, k);
                if (k < nz) {
                    double mx = o->mfx[w] + o->msx[w] / nsub, my = o->mfy[w] + o->msy[w] / nsub;
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, phi, i - 3 + m, j, k);
                    F[0][w] = mx * (C->scal_adv <= 1 ? orc_weno5(q, sgn(mx), zf) : orc_interp(q, sgn(mx), C->scal_adv));
                    for (int m = 0; m < 6; ++m) q[m] = CV(o, phi, i, j - 3 + m, k);
                    F[1][w] = my * (C->scal_adv <= 1 ? orc_weno5(q, sgn(my), zf) : orc_interp(q, sgn(my), C->scal_adv));
                }
                if (k == 0 || k == nz) { F[2][w] = 0.0; continue; }
                double mz = o->rom[w] + o->msz[w] / nsub;
                for (int m = 0; m < 6; ++m) q[m] = CV(o, phi, i, j, k - 3 + m);
                F[2][w] = mz * (C->scal_adv <= 1 ? orc_weno5(q, sgn(mz), zf) : orc_interp(q, sgn(mz), C->scal_adv));
            }
    #pragma omp parallel for
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX(o, i, j, k);
                double div = (F[0][IX(o, i + 1, j, k)] - F[0][c]) / dx
                           + (F[1][IX(o, i, j + 1, k)] - F[1][c]) / dy
                           + (F[2][IX(o, i, j, k + 1)] - F[2][c]);
                double v = sn_q[c] + adt * (-div / o->Hc[c] + (src ? src[c] : 0.0));
                rq[c] = (clip && v < 0.0) ? 0.0 : v;
            }
    free(phi); free(F[0]); free(F[1]); free(F[2]);
}
static void tracer_stage(orc *o, const double *rho_t, double adt, int nsub) {
    scalar_stage(o, o->rphi, o->sn_phi, NULL, 0, rho_t, adt, nsub);
}
static void tke_stage(orc *o, const double *rho_t, double adt, int nsub) {
    scalar_stage(o, o->rtke, o->sn_tke, o->tke_src, 1, rho_t, adt, nsub);
}

/* ------------------------------------------------------------------ Kessler microphysics (Sec. 2.4) */
/* Saturation mixing ratio over liquid water, q_vs = (R_d/R_v) e_s / (p - e_s), with the Tetens
 * (1930) vapour pressure e_s = 610.78 exp(17.27 (T - 273.16) / (T - 35.86)) Pa (reading: the paper's
 * Flatau et al. polynomial is cited, not printed; WRF's Kessler scheme uses this Tetens form). */
double orc_qvs(double T, double p) {
    double es = 610.78 * exp(17.27 * (T - 273.16) / (T - 35.86));
    return (ORC_RD / ORC_RV) * es / (p - es);
}
/* Rain terminal velocity of Klemp & Wilhelmson (1978), V = 3634 (rho q_r)^0.1346 (rho_0/rho)^(1/2)
 * cm/s with rho q_r in g/cm^3, rho_0 the base-state density at the ground: in SI units
 * V = 36.34 (1e-3 rho q_r)^0.1346 sqrt(rho_0 / rho) m/s. */
double orc_rain_speed(double rho, double qr, double rho_sfc) {
    if (!(qr > 0.0)) return 0.0;
    return 36.34 * pow(1.0e-3 * rho * qr, 0.1346) * sqrt(rho_sfc / rho);
}
/* Rain evaporation rate of Klemp & Wilhelmson (1978) [1/s]:
 *   E_r = (1/rho) (1 - q_v/q_vs) C (rho q_r)^0.525 / (5.4e5 + 2.55e6 / (p q_vs)),
 *   C = 1.6 + 124.9 (rho q_r)^0.2046, rho in g/cm^3, p in mb; 0 in saturated air or without rain. */
double orc_rain_evap(double rho, double qv, double qr, double qvs, double p) {
    if (!(qr > 0.0) || !(qv < qvs)) return 0.0;
    double rg = 1.0e-3 * rho, X = rg * qr;
    double C = 1.6 + 124.9 * pow(X, 0.2046);
    return (1.0 / rg) * (1.0 - qv / qvs) * C * pow(X, 0.525) / (5.4e5 + 2.55e6 / ((1.0e-2 * p) * qvs));
}
/* One time-split Kessler step (Kessler 1969; Klemp & Wilhelmson 1978) after the RK3 step, per
 * column, with the dry density unchanged:
 *   1. rain falls one explicit upwind step, F = rho q_r V through each cell's bottom face; what
 *      leaves the lowest cell adds F dt / rho_water to the surface accumulation;
 *   2. autoconversion k1 (q_c - a)^+ (k1 = 1e-3 1/s, a = 1e-3) and accretion k2 q_c q_r^0.875
 *      (k2 = 2.2 1/s) move cloud water to rain, at most all of it;
 *   3. saturation adjustment in one linearised step (Soong & Ogura 1973):
 *      s = (q_v - q_vs) / (1 + q_vs L_v 4098.17 / (c_p (T - 35.86)^2)), the Tetens slope at T = theta pi;
 *      condensation s (> 0) or evaporation of cloud water (at most q_c); rain evaporates
 *      min(dt E_r, (-s - q_c)^+, q_r), only what cloud water cannot cover;
 *      theta += L_v / (c_p pi) (condensation - evaporation), pi from the moist EOS before the step. */
static void kessler(orc *o) {
    const double dt = o->c.dt;
    int nx = o->nx, ny = o->ny, nz = o->nz;
#pragma omp parallel
    {
    double *F = dalloc(nz + 1);
#pragma omp for
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c0 = IX(o, i, j, 0);
            double rho_sfc = o->rho0[c0] / (1.0 + o->qv0[c0]);
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k);
                F[k] = o->rq[2][c] * orc_rain_speed(o->rho[c], o->rq[2][c] / o->rho[c], rho_sfc);
            }
            F[nz] = 0.0;
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k);
                o->rq[2][c] += dt * (F[k + 1] - F[k]) / o->Hc[c];
            }
            o->precip[(size_t)j * nx + i] += dt * F[0] / ORC_RHOW;
            for (int k = 0; k < nz; ++k) {
                size_t c = IX(o, i, j, k);
                double r = o->rho[c], th = o->rt[c] / r;
                double qv = o->rq[0][c] / r, qc = o->rq[1][c] / r, qr = o->rq[2][c] / r;
                double p, pie;
                eos_q(o->rt[c], qv, &p, &pie);
                double ar = 1.0e-3 * (qc - 1.0e-3);
                if (ar < 0.0) ar = 0.0;
                double cr = (qr > 0.0) ? 2.2 * qc * pow(qr, 0.875) : 0.0;
                double prod = dt * (ar + cr);
                if (prod > qc) prod = qc;
                qc -= prod;                 /* the cloud and rain the adjustment below sees */
                qr += prod;
                double T = th * pie;
                double qvs = orc_qvs(T, p);
                double sadj = (qv - qvs) / (1.0 + qvs * ORC_LV * 4098.17 / (ORC_CP * (T - 35.86) * (T - 35.86)));
                double ern = dt * orc_rain_evap(r, qv, qr, qvs, p);
                double lim = -sadj - qc;
                if (lim < 0.0) lim = 0.0;
                if (ern > lim) ern = lim;
                if (ern > qr) ern = qr;
                double cond = sadj > -qc ? sadj : -qc;
                /* increments of the conserved variables (nothing changes where nothing happens) */
                o->rt[c] += r * (ORC_LV / (ORC_CP * pie) * (cond - ern));
                o->rq[0][c] += r * (ern - cond);
                o->rq[1][c] += r * (cond - prod);
                o->rq[2][c] += r * (prod - ern);
                (void)th;
            }
        }
    free(F);
    }
}
/* test hook: one Kessler step on the current state */
int orc_kessler(orc *o) { kessler(o); return 0; }

/* ------------------------------------------------------------------ RK3 step (Sec. 3.1) */
static double *field_ptr(orc *o, int f) {
    switch (f) {
    case F_RHO: return o->rho;
    case F_RT: return o->rt;
    case F_RU: return o->ru;
    case F_RV: return o->rv;
    case F_RW: return o->rw;
    }
    return NULL;
}
static size_t field_len(const orc *o, int f) { return f == F_RW ? o->nw : o->ncell; }

static void rk3_step(orc *o) {
    const orc_cfg *C = &o->c;
    double dt = C->dt;
    int ns = C->n_substeps;
    apply_wall_bc(o, o->rw, o->ru, o->rv);
    for (int f = 0; f < 5; ++f) memcpy(o->sn[f], field_ptr(o, f), sizeof(double) * field_len(o, f));
    if (C->tracer) memcpy(o->sn_phi, o->rphi, sizeof(double) * o->ncell);
    int tke = (C->closure == 4);
    if (tke) memcpy(o->sn_tke, o->rtke, sizeof(double) * o->ncell);
    if (C->moist)
        for (int q = 0; q < 3; ++q) memcpy(o->sn_q[q], o->rq[q], sizeof(double) * o->ncell);
    const double alpha[3] = {1.0 / 3.0, 0.5, 1.0};
    /* S^t is held in o->rho.. (the state arrays), updated in place at the end of each stage */
    for (int s = 0; s < 3; ++s) {
        slow_rhs(o, o->rho, o->rt, o->ru, o->rv, o->rw);
        if (C->tracer || tke || C->moist) {
            memset(o->msx, 0, sizeof(double) * o->ncell);
            memset(o->msy, 0, sizeof(double) * o->ncell);
            memset(o->msz, 0, sizeof(double) * o->nw);
        }
        if (C->substep_mode == 1) {
            if (C->tracer) tracer_stage(o, o->rho, alpha[s] * dt, 1);
            if (tke) tke_stage(o, o->rho, alpha[s] * dt, 1);
            if (C->moist)
                for (int q = 0; q < 3; ++q) scalar_stage(o, o->rq[q], o->sn_q[q], o->q_src[q], 1, o->rho, alpha[s] * dt, 1);
            /* no substepping: S^(s) = S^n + alpha_s dt f(S^t) */
            for (int f = 0; f < 5; ++f) {
                double *S = field_ptr(o, f);
                for (size_t n = 0; n < field_len(o, f); ++n) S[n] = o->sn[f][n] + alpha[s] * dt * o->R[f][n];
            }
            apply_wall_bc(o, o->rw, o->ru, o->rv);
            continue;
        }
        /* substep schedule: stage 1 one substep of dt/3, stages 2, 3 ns/2 and ns substeps of dt/ns */
        int nsub = (s == 0) ? 1 : (s == 1 ? ns / 2 : ns);
        double dtau = (s == 0) ? dt / 3.0 : dt / ns;
        /* perturbations start from S^n - S^t (reading R9) */
        for (int f = 0; f < 5; ++f) {
            double *S = field_ptr(o, f);
            for (size_t n = 0; n < field_len(o, f); ++n) o->X[f][n] = o->sn[f][n] - S[n];
        }
        memcpy(o->Tprev, o->X[F_RT], sizeof(double) * o->ncell);
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i)
                for (int k = 0; k <= o->nz; ++k) {
                    size_t w = IX(o, i, j, k);
                    o->Om[w] = (k == 0 || k == o->nz) ? 0.0
                             : o->X[F_RW][w] - metric_shift(o, o->X[F_RU], o->X[F_RV], i, j, k);
                }
        /* stage-t fields used by the substeps: rho^t, Theta^t (pi^t, theta^t are in o->pi, o->th) */
        double *rho_t = dalloc(o->ncell), *rt_t = dalloc(o->ncell);
        memcpy(rho_t, o->rho, sizeof(double) * o->ncell);
        memcpy(rt_t, o->rt, sizeof(double) * o->ncell);
        for (int n = 0; n < nsub; ++n) substep(o, rho_t, rt_t, dtau);
        if (C->tracer) tracer_stage(o, rho_t, alpha[s] * dt, nsub);
        if (tke) tke_stage(o, rho_t, alpha[s] * dt, nsub);
        if (C->moist)
            for (int q = 0; q < 3; ++q) scalar_stage(o, o->rq[q], o->sn_q[q], o->q_src[q], 1, rho_t, alpha[s] * dt, nsub);
        free(rho_t); free(rt_t);
        /* S^(s) = S^t + X'' */
        for (int f = 0; f < 5; ++f) {
            double *S = field_ptr(o, f);
            for (size_t n = 0; n < field_len(o, f); ++n) S[n] += o->X[f][n];
        }
    }
    if (C->moist) kessler(o);   /* microphysics after the dycore step (time split) */
}

/* ------------------------------------------------------------------ public API (ctypes) */
/* Initial state from a potential-temperature perturbation at unchanged pressure (Sec. 4.1.2:
 * warm perturbations at constant pressure give negative density perturbations):
 *   theta = theta0 + dtheta, rho theta = rho0 theta0, rho = rho theta / theta;
 * velocities given at faces are multiplied by the face-averaged density; walls get Omega = 0. */
void orc_set_initial_q(orc *o, const double *dtheta, const double *qv, const double *u, const double *v,
                       const double *w);
void orc_set_initial(orc *o, const double *dtheta, const double *u, const double *v, const double *w) {
    orc_set_initial_q(o, dtheta, NULL, u, v, w);
}
/* Moist configurations take the water vapour q_v at cells (NULL: the base state's q_v0) and keep
 * the pressure too: rho_d theta_d (1 + (R_v/R_d) q_v) = rho_d0 theta0 (1 + (R_v/R_d) q_v0), with
 * rho_d0 = rho0 / (1 + q_v0) the base dry density; rho q_c = rho q_r = 0.  Every field's initial
 * value becomes the reference of the lateral relaxation zones. */
void orc_set_initial_q(orc *o, const double *dtheta, const double *qv, const double *u, const double *v,
                       const double *w) {
    const double ev = ORC_RV / ORC_RD;
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                size_t c = IX(o, i, j, k);
                double th = o->th0[c] + (dtheta ? dtheta[c] : 0.0);
                if (o->c.anelastic) {          /* Sec. 2.2: the density is the base density */
                    o->rho[c] = o->rho0[c];
                    o->rt[c] = o->rho0[c] * th;
                } else if (o->c.moist) {
                    double q0 = o->qv0[c], q = qv ? qv[c] : q0;
                    double rd0 = o->rho0[c] / (1.0 + q0), f = (1.0 + ev * q0) / (1.0 + ev * q);
                    o->rt[c] = rd0 * o->th0[c] * f;
                    o->rho[c] = rd0 * (o->th0[c] / th) * f;   /* the dry form times f (1 without vapour) */
                    o->rq[0][c] = o->rho[c] * q;
                    o->rq[1][c] = 0.0;
                    o->rq[2][c] = 0.0;
                } else {
                    o->rt[c] = o->rho0[c] * o->th0[c];
                    o->rho[c] = o->rho0[c] * (o->th0[c] / th);   /* = rho0 theta0 / theta; exact at rest */
                }
            }
    for (int k = 0; k <= o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                size_t c = IX(o, i, j, k);
                if (k < o->nz) {
                    o->ru[c] = u ? u[c] * 0.5 * (o->rho[IX(o, i - 1, j, k)] + o->rho[c]) : 0.0;
                    o->rv[c] = v ? v[c] * 0.5 * (o->rho[IX(o, i, j - 1, k)] + o->rho[c]) : 0.0;
                }
                o->rw[c] = w ? w[c] * 0.5 * (CV(o, o->rho, i, j, k - 1) + CV(o, o->rho, i, j, k)) : 0.0;
            }
    apply_wall_bc(o, o->rw, o->ru, o->rv);
    o->have_state = 1;
    for (int f = 0; f < 5; ++f) memcpy(o->ref[f], field_ptr(o, f), sizeof(double) * field_len(o, f));
    for (int q = 0; q < 3; ++q) memcpy(o->ref_q[q], o->rq[q], sizeof(double) * o->ncell);
}
/* the current state becomes the reference of the lateral relaxation zones */
int orc_capture_reference(orc *o) {
    for (int f = 0; f < 5; ++f) memcpy(o->ref[f], field_ptr(o, f), sizeof(double) * field_len(o, f));
    for (int q = 0; q < 3; ++q) memcpy(o->ref_q[q], o->rq[q], sizeof(double) * o->ncell);
    return 0;
}
/* accumulated surface precipitation [m of liquid water] per column (ny*nx) */
int orc_get_precip(orc *o, double *dst) {
    memcpy(dst, o->precip, sizeof(double) * (size_t)o->nx * o->ny);
    return 0;
}

/* fields 0..4 = rho, rho theta, rho u, rho v, rho w; 5..7 = base rho0, p0, theta0 (get only);
 * 8 = rho phi (passive scalar); 9 = rho e (Deardorff); 10..12 = rho q_v, rho q_c, rho q_r;
 * 13 = base q_v0 (get only) */
/* passive-scalar initial state: rho phi = rho phi0 at cells, with the current rho */
int orc_set_tracer_initial(orc *o, const double *phi) {
    for (size_t c = 0; c < o->ncell; ++c) o->rphi[c] = o->rho[c] * phi[c];
    return 0;
}
int orc_get_field(orc *o, int f, double *dst) {
    if (f >= 0 && f < 5) { memcpy(dst, field_ptr(o, f), sizeof(double) * field_len(o, f)); return 0; }
    if (f == 5) { memcpy(dst, o->rho0, sizeof(double) * o->ncell); return 0; }
    if (f == 6) { memcpy(dst, o->p0, sizeof(double) * o->ncell); return 0; }
    if (f == 7) { memcpy(dst, o->th0, sizeof(double) * o->ncell); return 0; }
    if (f == 8) { memcpy(dst, o->rphi, sizeof(double) * o->ncell); return 0; }
    if (f == 9) { memcpy(dst, o->rtke, sizeof(double) * o->ncell); return 0; }
    if (f >= 10 && f <= 12) { memcpy(dst, o->rq[f - 10], sizeof(double) * o->ncell); return 0; }
    if (f == 13) { memcpy(dst, o->qv0, sizeof(double) * o->ncell); return 0; }
    if (f == 14) { memcpy(dst, o->pa, sizeof(double) * o->ncell); return 0; }
    return -1;
}
int orc_set_field(orc *o, int f, const double *src) {
    if (f == 8) { memcpy(o->rphi, src, sizeof(double) * o->ncell); return 0; }
    if (f == 9) { memcpy(o->rtke, src, sizeof(double) * o->ncell); return 0; }
    if (f >= 10 && f <= 12) { memcpy(o->rq[f - 10], src, sizeof(double) * o->ncell); return 0; }
    if (f == 14) { memcpy(o->pa, src, sizeof(double) * o->ncell); return 0; }
    if (f < 0 || f >= 5) return -1;
    memcpy(field_ptr(o, f), src, sizeof(double) * field_len(o, f));
    o->have_state = 1;
    return 0;
}
/* geometry: 0 zc, 1 Hc, 2 Hx, 3 Hy, 4 hxi_x, 5 heta_y (cells); 6 zw, 7 hxi_w, 8 heta_w, 9 zn (w levels) */
int orc_get_geom(orc *o, int which, double *dst) {
    double *src[] = {o->zc, o->Hc, o->Hx, o->Hy, o->hxi_x, o->heta_y, o->zw, o->hxi_w, o->heta_w, o->zn};
    if (which < 0 || which > 9) return -1;
    memcpy(dst, src[which], sizeof(double) * (which < 6 ? o->ncell : o->nw));
    return 0;
}
/* the model of the learned closure (closure 3); it must be set before the first step */
int orc_set_sgs_model(orc *o, void (*fn)(void *, const double *, const double *, const double *, const double *,
                                         const double *, double *), void *user) {
    if (!o->sgs_planes) o->sgs_planes = dalloc(9 * o->ncell);
    o->sgs_model = fn;
    o->sgs_user = user;
    return 0;
}
int orc_step(orc *o, int nsteps) {
    if (!o->have_state) return -5;
    if (o->c.anelastic) return -6;     /* the anelastic steps are driven from oracle/anelastic.py */
    if (o->c.closure == 3 && !o->sgs_model) return -5;
    for (int n = 0; n < nsteps; ++n) rk3_step(o);
    return 0;
}
/* slow tendencies of the current state (no time advance): R_rho, R_Theta, R_U, R_V, R_W, and
 * the EOS fields p', pi, theta */
int orc_slow_rhs(orc *o, double *Rr, double *Rt, double *Ru, double *Rv, double *Rw,
                 double *pp, double *pi, double *th) {
    if (o->c.closure == 3 && !o->sgs_model) return -5;
    slow_rhs(o, o->rho, o->rt, o->ru, o->rv, o->rw);
    memcpy(Rr, o->R[F_RHO], sizeof(double) * o->ncell);
    memcpy(Rt, o->R[F_RT], sizeof(double) * o->ncell);
    memcpy(Ru, o->R[F_RU], sizeof(double) * o->ncell);
    memcpy(Rv, o->R[F_RV], sizeof(double) * o->ncell);
    memcpy(Rw, o->R[F_RW], sizeof(double) * o->nw);
    if (pp) memcpy(pp, o->pp, sizeof(double) * o->ncell);
    if (pi) memcpy(pi, o->pi, sizeof(double) * o->ncell);
    if (th) memcpy(th, o->th, sizeof(double) * o->ncell);
    return 0;
}
/* One acoustic substep on given perturbations (test hook): the current state is the stage
 * state S^t; X[0..4] = rho'', Theta'', U'', V'', W'' in/out; R[0..4] the slow tendencies
 * (NULL = zero).  Theta'' of the previous substep is taken equal to the given one. */
int orc_substep_once(orc *o, double dtau, double *Xr, double *Xt, double *Xu, double *Xv, double *Xw,
                     const double *Rr, const double *Rt, const double *Ru, const double *Rv, const double *Rw) {
    double *X[5] = {Xr, Xt, Xu, Xv, Xw};
    const double *R[5] = {Rr, Rt, Ru, Rv, Rw};
    eos_pass(o, o->rho, o->rt);
    for (int f = 0; f < 5; ++f) {
        size_t n = field_len(o, f);
        memcpy(o->X[f], X[f], sizeof(double) * n);
        if (R[f]) memcpy(o->R[f], R[f], sizeof(double) * n);
        else memset(o->R[f], 0, sizeof(double) * n);
    }
    memcpy(o->Tprev, o->X[F_RT], sizeof(double) * o->ncell);
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i)
            for (int k = 0; k <= o->nz; ++k) {
                size_t w = IX(o, i, j, k);
                o->Om[w] = (k == 0 || k == o->nz) ? 0.0
                         : o->X[F_RW][w] - metric_shift(o, o->X[F_RU], o->X[F_RV], i, j, k);
            }
    substep(o, o->rho, o->rt, dtau);
    for (int f = 0; f < 5; ++f) memcpy(X[f], o->X[f], sizeof(double) * field_len(o, f));
    return 0;
}

/* eddy viscosity of the last slow-RHS evaluation */
int orc_get_mu(orc *o, double *dst) { memcpy(dst, o->mu, sizeof(double) * o->ncell); return 0; }
/* cell arrays of the last slow-RHS evaluation: 0 mu (= rho K_m), 1 rho K_h (Deardorff),
 * 2 the SGS-energy source rho (P + B - eps) + div(2 mu grad e) (Deardorff) */
int orc_get_aux(orc *o, int which, double *dst) {
    const double *src[] = {o->mu, o->muh, o->tke_src};
    if (which < 0 || which > 2) return -1;
    memcpy(dst, src[which], sizeof(double) * o->ncell);
    return 0;
}
/* domain-integrated mass: sum of rho times the physical cell volume, in fixed (k,j,i) order.  The
 * sum is compensated (Neumaier's variant of Kahan summation: the rounding error of every addition
 * is carried and added at the end), so its error does not grow with the cell count: a plain
 * running sum over millions of cells rounds by ~1e-11 relative, more than the drift it measures. */
double orc_mass(orc *o) {
    double s = 0.0, comp = 0.0;
    for (size_t c = 0; c < o->ncell; ++c) {
        const double x = o->rho[c] * o->Hc[c] * o->c.dx * o->c.dy;
        const double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x;
        else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}
int orc_sizeof_cfg(void) { return (int)sizeof(orc_cfg); }

/* thread count of the OpenMP loops (results do not depend on it) */
#include <omp.h>
void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int orc_get_threads(void) { return omp_get_max_threads(); }
