// C ABI of the dycore library (declared in include/erf.h): argument checks, workspace carving,
// init (metrics of App. B, HSE base state of Sec. 3.8), state I/O, and the RK3 step of Sec. 3.1
// captured once as a CUDA graph and replayed per step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/erf.h"
#include "erf_dev.cuh"
#include "erf_launch.h"
#include "erf_mixed.h"
#include "erf_closure.h"

using namespace erfk;

namespace {

struct Carve {
    char *base;
    size_t off, cap;
    bool dry;   // size-only pass
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = dry ? nullptr : reinterpret_cast<T *>(base + off);
        off += n * sizeof(T);
        return p;
    }
};

thread_local std::string g_init_error;

}  // namespace

struct erf_handle {
    erf_grid_desc grid;
    erf_config cfg;
    Geo geo;
    Phys ph;
    cudaStream_t user = nullptr;   // caller's stream
    cudaStream_t cap = nullptr;    // private stream used for graph capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_step = 0;
    bool have_state = false;
    long long steps_done = 0;
    std::string err;
    // workspace arrays
    double *hn, *hc, *hxf, *hyf, *gxh, *gyh, *g4xq, *g4yq;
    double *dzeta, *zetac, *s, *sc, *ds, *dzc, *delta2, *rdzeta, *rdzc, *knz, *knt, *delta;
    double *rho0, *th0, *p0;
    double *rH3 = nullptr, *rHx3 = nullptr, *rHy3 = nullptr, *rdzw3 = nullptr, *rdz2 = nullptr;
    double *Hx3 = nullptr, *Hy3 = nullptr;
    // passive scalar (FP64 path): rho phi (stage state), its S^n copy, substep flux sums
    double *tphi = nullptr, *snphi = nullptr, *msx = nullptr, *msy = nullptr, *msz = nullptr;
    // Deardorff closure (FP64 path): rho e (stage state), its S^n copy, the stage's energy source
    // and the heat diffusivity rho K_h
    double *tke = nullptr, *sntke = nullptr, *tke_src = nullptr, *muh = nullptr;
    // moisture (FP64 path): rho q_v, rho q_c, rho q_r (stage state), their S^n copies, their
    // slow-pass sources, the base-state q_v0, the sounding knots and the surface precipitation
    double *rq[3] = {nullptr, nullptr, nullptr}, *snq[3] = {nullptr, nullptr, nullptr};
    double *qsrc[3] = {nullptr, nullptr, nullptr}, *qv0 = nullptr, *qkz = nullptr, *qkv = nullptr;
    double *precip = nullptr;
    // lateral relaxation zones: the reference state (rho, rho theta, rho u, rho v, rho w, rho q's)
    double *ref[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // anelastic equation set: projection pressure p' (now, at the step start, after stage 1), FFT
    // twiddles and second-difference eigenvalues
    double *pa = nullptr, *pan = nullptr, *pa1 = nullptr, *lamx = nullptr, *lamy = nullptr;
    double2 *twx = nullptr, *twy = nullptr;
    F5 st, sn, x, R;
    double *pp, *pi, *th, *Tp, *Om;
    Tri tri;
    TriM mtri;
    double *mstage = nullptr;
    double *ux, *vy, *wz, *mfx, *mfy, *rom, *mu, *flux;
    double *diag_part, *diag_out;
    // mixed-precision path (flat grids): FP32 perturbation fields + FP64 solve scratch
    bool mixed = false;
    F5f mst, msn, mx, mR;
    float *mpp, *mpi, *mthp, *mTp, *mux, *mvy, *mwz, *mmfx, *mmfy, *mmu, *mbase;
    double *mdbuf, *mrt0;
    float *mflux = nullptr;                 // slow-tendency face fluxes (3 planes of nw)
    MxTma tma{};                            // TMA tile maps of the stencil fields
    bool tma_enabled = true;
    int column_fusion = -1;                 // ERF_OPT_COLUMN_FUSION: -1 by column count, 0 off, 1 on
    int warp_columns = -1;                  // ERF_OPT_WARP_COLUMNS: -1 by column count, 0 off, 1 on
    unsigned *kerr = nullptr;               // set by a kernel whose bounded wait gave up
    float *mX0 = nullptr, *mY0 = nullptr;   // beta-weighted Theta'', rho'' of the vertical substep (in mflux)
    // passive scalar (mixed path, FP32): rho phi, its S^n copy, substep momentum sums
    float *mtphi = nullptr, *msnphi = nullptr;
    TrSum mms{nullptr, nullptr, nullptr};
    MxBase mb;
    // learned closure
    void *cl_w = nullptr;
    float *cl_b = nullptr, *cl_stats = nullptr, *cl_blob = nullptr, *cl_out = nullptr;
    unsigned *cl_nfb = nullptr;
    bool cl_ready = false;
};

// TMA tile maps of the mixed path's stencil fields (theta' and the face velocities)
static bool mx_encode_tiles(erf_handle *h) {
    const Geo &g = h->geo;
    return mx_encode_cell_tile_map(&h->tma.thp, h->mthp, g, g.nz) && mx_encode_cell_tile_map(&h->tma.ux, h->mux, g, g.nz) &&
           mx_encode_cell_tile_map(&h->tma.vy, h->mvy, g, g.nz) && mx_encode_cell_tile_map(&h->tma.wz, h->mwz, g, g.nz + 1);
}

static erf_status fail(erf_handle *h, erf_status st, const std::string &msg) {
    if (h) h->err = msg;
    else g_init_error = msg;
    return st;
}
static erf_status cuda_fail(erf_handle *h, cudaError_t e, const char *where) {
    return fail(h, ERF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static erf_status validate(const erf_grid_desc *g, const erf_config *c, std::string &msg) {
    if (!g || !c) { msg = "NULL grid or config"; return ERF_EINVAL; }
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nz > ERF_NZ_MAX) { msg = "grid sizes out of range"; return ERF_EINVAL; }
    if ((long long)g->nx * g->ny * (g->nz + 1) >= (1LL << 31) || g->ny > 65535) {
        msg = "grid too large: nx*ny*(nz+1) must be below 2^31 and ny at most 65535";
        return ERF_EINVAL;
    }
    if (!(g->dx > 0.0) || !(g->dy > 0.0)) { msg = "dx, dy must be positive"; return ERF_EINVAL; }
    if (!g->z_faces) { msg = "z_faces is NULL"; return ERF_EINVAL; }
    if (g->z_faces[0] != 0.0) { msg = "z_faces[0] must be 0"; return ERF_EINVAL; }
    for (int k = 0; k < g->nz; ++k)
        if (!(g->z_faces[k + 1] > g->z_faces[k])) { msg = "z_faces must increase"; return ERF_EINVAL; }
    if (g->terrain_nodes && g->terrain_beta < 0) { msg = "terrain_beta must be >= 0"; return ERF_EINVAL; }
    if (!(c->dt > 0.0)) { msg = "dt must be positive"; return ERF_EINVAL; }
    if (c->substep_mode != 0 && c->substep_mode != 1) { msg = "substep_mode must be 0 or 1"; return ERF_EINVAL; }
    if (c->substep_mode == 0 && (c->n_substeps < 2 || c->n_substeps % 2)) { msg = "n_substeps must be even and >= 2"; return ERF_EINVAL; }
    if (c->closure < 0 || c->closure > 4) { msg = "closure out of range"; return ERF_EINVAL; }
    if (c->closure == 4 && c->precision != ERF_PREC_FP64) {
        msg = "the Deardorff closure runs on the FP64 path";
        return ERF_EUNSUPPORTED;
    }
    if (c->ray_fields < 0 || c->ray_fields > 15 || !(c->ray_tau >= 0.0) || !(c->ray_zd >= 0.0) ||
        (c->ray_fields != 0 && !(c->ray_zd < g->z_faces[g->nz]))) {
        msg = "Rayleigh damping: fields 0..15, tau >= 0, 0 <= z_d < domain top";
        return ERF_EINVAL;
    }
    if (c->anelastic != 0 && c->anelastic != 1) { msg = "anelastic must be 0 or 1"; return ERF_EINVAL; }
    if (c->anelastic) {
        auto pow2 = [](int n) { return n >= 1 && n <= 4096 && (n & (n - 1)) == 0; };
        if (c->precision != ERF_PREC_FP64 || c->moist || c->tracer || c->closure == 4 || c->relax_tau > 0.0) {
            msg = "the anelastic equation set runs on the FP64 path without moisture, scalars or relaxation zones";
            return ERF_EUNSUPPORTED;
        }
        if (!pow2(g->nx) || !pow2(g->ny)) {
            msg = "the anelastic projection's FFT needs nx and ny powers of two up to 4096";
            return ERF_EUNSUPPORTED;
        }
        if (g->terrain_nodes)
            for (long long n = 0; n < (long long)g->nx * g->ny; ++n)
                if (g->terrain_nodes[n] != 0.0) { msg = "the anelastic projection is built for flat grids"; return ERF_EUNSUPPORTED; }
    }
    if (c->moist != 0 && c->moist != 1) { msg = "moist must be 0 or 1"; return ERF_EINVAL; }
    if (c->moist && c->precision != ERF_PREC_FP64) {
        msg = "moisture and microphysics run on the FP64 path";
        return ERF_EUNSUPPORTED;
    }
    if (c->moist && (c->n_qknots < 1 || !c->qknot_z || !c->qknot_v)) {
        msg = "a moist configuration needs its water-vapour sounding (n_qknots >= 1)";
        return ERF_EINVAL;
    }
    if (!(c->relax_tau >= 0.0) || (c->relax_tau > 0.0 && !(c->relax_width > 0.0))) {
        msg = "relaxation zones: relax_tau >= 0 and relax_width > 0";
        return ERF_EINVAL;
    }
    if (c->relax_tau > 0.0 && c->precision != ERF_PREC_FP64) {
        msg = "relaxation zones run on the FP64 path";
        return ERF_EUNSUPPORTED;
    }
    if (c->ray_fields != 0 && c->ray_tau > 0.0 && c->precision != ERF_PREC_FP64) {
        msg = "Rayleigh damping runs on the FP64 path";
        return ERF_EUNSUPPORTED;
    }
    if (c->closure == 3 && c->precision != ERF_PREC_MIXED32) {
        msg = "the learned closure runs on the mixed-precision path";
        return ERF_EUNSUPPORTED;
    }
    if (c->scal_adv != 0 && c->scal_adv != 1 && c->scal_adv != 3) { msg = "scal_adv must be 0, 1 or 3"; return ERF_EINVAL; }
    if (c->mom_adv != 0 && c->mom_adv != 3 && c->mom_adv != 5) { msg = "mom_adv must be 0, 3 or 5"; return ERF_EINVAL; }
    if (c->surface < 0 || c->surface > 1) { msg = "surface out of range"; return ERF_EINVAL; }
    if (c->precision != ERF_PREC_FP64 && c->precision != ERF_PREC_MIXED32) { msg = "precision out of range"; return ERF_EINVAL; }
    if (c->n_knots < 0 || (c->n_knots > 0 && (!c->knot_z || !c->knot_theta))) { msg = "bad sounding knots"; return ERF_EINVAL; }
    if (c->closure == ERF_CLOSURE_SMAGORINSKY && !(c->Cs >= 0.0)) { msg = "Cs must be >= 0"; return ERF_EINVAL; }
    if ((c->closure != 0) && !(c->Pr_t > 0.0)) { msg = "Pr_t must be positive"; return ERF_EINVAL; }
    if (c->surface == ERF_SURFACE_MOST && !(c->z0 > 0.0)) { msg = "z0 must be positive"; return ERF_EINVAL; }
    bool terr = false;
    if (g->terrain_nodes)
        for (long long n = 0; n < (long long)g->nx * g->ny; ++n)
            if (g->terrain_nodes[n] != 0.0) { terr = true; break; }
    if (terr && (c->closure != 0 || c->surface != 0)) {
        msg = "subgrid closure / MOST over terrain is not supported (flat grids only)";
        return ERF_EUNSUPPORTED;
    }
    if (c->tracer != 0 && c->tracer != 1) { msg = "tracer must be 0 or 1"; return ERF_EINVAL; }
    if (terr && c->precision == ERF_PREC_MIXED32) {
        msg = "the mixed-precision path is built for flat grids only";
        return ERF_EUNSUPPORTED;
    }
    return ERF_OK;
}

// lays out every array; with dry = true only sizes
static size_t carve(erf_handle *h, const erf_grid_desc *g, const erf_config *c, void *ws, bool dry) {
    Carve cv{reinterpret_cast<char *>(ws), 0, 0, dry};
    long long nx = g->nx, ny = g->ny, nz = g->nz;
    long long nxy = nx * ny, nc = nxy * nz, nw = nxy * (nz + 1);
    erf_handle tmp;
    erf_handle *H = h ? h : &tmp;
    H->hn = cv.take<double>(nxy); H->hc = cv.take<double>(nxy); H->hxf = cv.take<double>(nxy);
    H->hyf = cv.take<double>(nxy); H->gxh = cv.take<double>(nxy); H->gyh = cv.take<double>(nxy);
    H->g4xq = cv.take<double>(nxy); H->g4yq = cv.take<double>(nxy);
    H->dzeta = cv.take<double>(nz); H->zetac = cv.take<double>(nz); H->s = cv.take<double>(nz + 1);
    H->sc = cv.take<double>(nz); H->ds = cv.take<double>(nz); H->dzc = cv.take<double>(nz + 1);
    H->delta2 = cv.take<double>(nz);
    H->rdzeta = cv.take<double>(nz);
    H->rdzc = cv.take<double>(nz + 1);
    H->delta = cv.take<double>(nz);
    H->knz = cv.take<double>(c->n_knots > 0 ? c->n_knots : 1);
    H->knt = cv.take<double>(c->n_knots > 0 ? c->n_knots : 1);
    bool terr = false;
    if (g->terrain_nodes)
        for (long long n = 0; n < nxy; ++n) if (g->terrain_nodes[n] != 0.0) { terr = true; break; }
    long long nb = terr ? nc : nz;
    H->rho0 = cv.take<double>(nb); H->th0 = cv.take<double>(nb); H->p0 = cv.take<double>(nb);
    if (c->precision == ERF_PREC_MIXED32) {
        H->mixed = true;
        F5f *sets[4] = {&H->mst, &H->msn, &H->mx, &H->mR};
        for (F5f *f : sets) {
            f->r = cv.take<float>(nc); f->t = cv.take<float>(nc); f->u = cv.take<float>(nc);
            f->v = cv.take<float>(nc); f->w = cv.take<float>(nw);
        }
        H->mpp = cv.take<float>(nc); H->mpi = cv.take<float>(nc); H->mthp = cv.take<float>(nc);
        H->mTp = cv.take<float>(nc);
        H->mux = cv.take<float>(nc); H->mvy = cv.take<float>(nc); H->mwz = cv.take<float>(nw);
        H->mmfx = cv.take<float>(nc); H->mmfy = cv.take<float>(nc);
        // eddy viscosity, then (eddy-viscosity closures) the three diagonal stresses
        H->mmu = cv.take<float>((c->closure == 1 || c->closure == 2) ? 4 * nc : nc);
        H->mbase = cv.take<float>(mx_base_floats((int)nz));
        H->mrt0 = cv.take<double>(nz);
        H->mdbuf = cv.take<double>(nw);
        // the flux planes are free during the substeps, which keep X0 and Y0 there
        H->mflux = cv.take<float>(3 * nw);
        H->mX0 = H->mflux; H->mY0 = H->mflux + nw;
        H->mstage = cv.take<double>(nw);   // FP64 staging outside the step; the stage's sub-diagonal during it
        H->mtri.a = reinterpret_cast<float *>(H->mstage); H->mtri.cp = cv.take<double>(nw); H->mtri.im = cv.take<double>(nw);
        H->mtri.P = cv.take<float>(nw); H->mtri.Q = cv.take<float>(nw);
        if (c->tracer) {
            H->mtphi = cv.take<float>(nc); H->msnphi = cv.take<float>(nc);
            H->mms.x = cv.take<float>(nc); H->mms.y = cv.take<float>(nc); H->mms.z = cv.take<float>(nw);
        }
        if (c->closure == 3) {
            H->cl_w = cv.take<unsigned short>(64 * 16 + 64 * 64 * 2 + 16 * 64);
            H->cl_b = cv.take<float>(64 * 3 + 16);
            H->cl_stats = cv.take<float>(2 * CL_NIN + 2 * CL_NOUT);
            H->cl_blob = cv.take<float>(CL_BLOB_FLOATS);
            H->cl_out = cv.take<float>(9 * nc);
            H->cl_nfb = cv.take<unsigned>(4);
        }
    } else {
    F5 *sets[4] = {&H->st, &H->sn, &H->x, &H->R};
    for (F5 *f : sets) {
        f->r = cv.take<double>(nc); f->t = cv.take<double>(nc); f->u = cv.take<double>(nc);
        f->v = cv.take<double>(nc); f->w = cv.take<double>(nw);
    }
    H->pp = cv.take<double>(nc); H->pi = cv.take<double>(nc); H->th = cv.take<double>(nc);
    H->Tp = cv.take<double>(nc); H->Om = cv.take<double>(nw);
    H->tri.a = cv.take<double>(nw); H->tri.cp = cv.take<double>(nw); H->tri.im = cv.take<double>(nw);
    H->tri.P = cv.take<double>(nw); H->tri.Q = cv.take<double>(nw);
    H->ux = cv.take<double>(nc); H->vy = cv.take<double>(nc); H->mfx = cv.take<double>(nc);
    H->mfy = cv.take<double>(nc); H->wz = cv.take<double>(nw); H->rom = cv.take<double>(nw);
    H->mu = cv.take<double>(nc);
    H->flux = cv.take<double>(3 * nw);   // theta, then each momentum component's fluxes (3 planes of nw)
    if (terr) {
        H->rH3 = cv.take<double>(nc); H->rHx3 = cv.take<double>(nc); H->rHy3 = cv.take<double>(nc);
        H->Hx3 = cv.take<double>(nc); H->Hy3 = cv.take<double>(nc);
        H->rdzw3 = cv.take<double>(nc); H->rdz2 = cv.take<double>(nc);
    }
    if (c->tracer) {
        H->tphi = cv.take<double>(nc); H->snphi = cv.take<double>(nc);
    }
    if (c->tracer || c->closure == 4 || c->moist) {
        H->msx = cv.take<double>(nc); H->msy = cv.take<double>(nc); H->msz = cv.take<double>(nw);
    }
    if (c->moist) {
        for (int q = 0; q < 3; ++q) {
            H->rq[q] = cv.take<double>(nc); H->snq[q] = cv.take<double>(nc); H->qsrc[q] = cv.take<double>(nc);
        }
        H->qv0 = cv.take<double>(nb);
        H->qkz = cv.take<double>(c->n_qknots); H->qkv = cv.take<double>(c->n_qknots);
        H->precip = cv.take<double>(nxy);
    }
    if (c->anelastic) {
        H->pa = cv.take<double>(nc); H->pan = cv.take<double>(nc); H->pa1 = cv.take<double>(nc);
        H->lamx = cv.take<double>(nx); H->lamy = cv.take<double>(ny);
        H->twx = cv.take<double2>(nx / 2 > 0 ? nx / 2 : 1); H->twy = cv.take<double2>(ny / 2 > 0 ? ny / 2 : 1);
    }
    if (c->relax_tau > 0.0) {
        for (int f = 0; f < 5; ++f) H->ref[f] = cv.take<double>(f == 4 ? nw : nc);
        if (c->moist)
            for (int q = 0; q < 3; ++q) H->ref[5 + q] = cv.take<double>(nc);
    }
    if (c->closure == 4) {
        H->tke = cv.take<double>(nc); H->sntke = cv.take<double>(nc);
        H->tke_src = cv.take<double>(nc); H->muh = cv.take<double>(nc);
    }
    }
    H->kerr = cv.take<unsigned>(4);
    H->diag_part = cv.take<double>(6 * DIAG_PARTS);
    H->diag_out = cv.take<double>(8);
    return cv.off + 256;
}

extern "C" erf_status erf_workspace_bytes(const erf_grid_desc *grid, const erf_config *cfg, size_t *bytes) {
    std::string msg;
    erf_status st = validate(grid, cfg, msg);
    if (st != ERF_OK) return fail(nullptr, st, msg);
    if (!bytes) return fail(nullptr, ERF_EINVAL, "bytes is NULL");
    *bytes = carve(nullptr, grid, cfg, nullptr, true);
    return ERF_OK;
}

static void fill_geo(erf_handle *h) {
    const erf_grid_desc &g = h->grid;
    Geo &G = h->geo;
    G.nx = g.nx; G.ny = g.ny; G.nz = g.nz;
    G.nxy = (long long)g.nx * g.ny; G.nc = G.nxy * g.nz; G.nw = G.nxy * (g.nz + 1);
    G.dx = g.dx; G.dy = g.dy; G.rdx = 1.0 / g.dx; G.rdy = 1.0 / g.dy;
    G.dzeta = h->dzeta; G.zetac = h->zetac; G.s = h->s; G.sc = h->sc; G.ds = h->ds; G.dzc = h->dzc;
    G.delta2 = h->delta2;
    G.rdzeta = h->rdzeta;
    G.rdzc = h->rdzc;
    G.delta = h->delta;
    G.hc = h->hc; G.hxf = h->hxf; G.hyf = h->hyf; G.gxh = h->gxh; G.gyh = h->gyh; G.g4xq = h->g4xq; G.g4yq = h->g4yq;
    G.rho0 = h->rho0; G.th0 = h->th0; G.p0 = h->p0;
    G.rH3 = h->rH3; G.rHx3 = h->rHx3; G.rHy3 = h->rHy3; G.rdzw3 = h->rdzw3; G.rdz2 = h->rdz2;
    G.Hx3 = h->Hx3; G.Hy3 = h->Hy3;
    const erf_config &c = h->cfg;
    Phys &P = h->ph;
    P.g = c.gravity; P.f_cor = c.f_cor; P.u_g = c.u_g; P.v_g = c.v_g; P.Cs = c.Cs; P.Pr_t = c.Pr_t; P.nu = c.nu;
    P.z0 = c.z0; P.Qs = c.sfc_theta_flux; P.beta_s = c.beta_s; P.beta_d = c.beta_d;
    P.rPr_t = 1.0 / c.Pr_t;
    P.b1 = 0.5 * (1.0 - c.beta_s);
    P.b2 = 0.5 * (1.0 + c.beta_s);
    P.closure = c.closure; P.surface = c.surface; P.scal_adv = c.scal_adv;
    P.mom3 = c.mom_adv == 3 ? 1 : 0;
    P.ray_tau = c.ray_tau;
    P.ray_zd = c.ray_zd;
    P.ray_fields = c.ray_tau > 0.0 ? c.ray_fields : 0;
    P.ray_zt = 0.0;   // set in erf_init_grid from the face heights
    P.moist = c.moist ? 1 : 0;
    P.rqv = h->rq[0]; P.rqc = h->rq[1]; P.rqr = h->rq[2];
    P.relax_tau = c.relax_tau;
    P.relax_w = c.relax_width;
    P.Lx = g.nx * g.dx;
    P.anelastic = c.anelastic ? 1 : 0;
    G.qv0 = h->qv0;
}

extern "C" erf_status erf_init_grid(const erf_grid_desc *grid, const erf_config *cfg, void *d_workspace,
                                    size_t workspace_bytes, void *cuda_stream, erf_handle **out) {
    std::string msg;
    erf_status vs = validate(grid, cfg, msg);
    if (vs != ERF_OK) return fail(nullptr, vs, msg);
    if (!out) return fail(nullptr, ERF_EINVAL, "out is NULL");
    if (!d_workspace) return fail(nullptr, ERF_EINVAL, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0) return fail(nullptr, ERF_EINVAL, "workspace must be 256-byte aligned");
    size_t need = carve(nullptr, grid, cfg, nullptr, true);
    if (workspace_bytes < need)
        return fail(nullptr, ERF_ENOSPACE, "workspace too small: need " + std::to_string(need) + " bytes");
    erf_handle *h = new (std::nothrow) erf_handle();
    if (!h) return fail(nullptr, ERF_EINVAL, "out of host memory");
    h->grid = *grid;
    h->grid.z_faces = nullptr;
    h->grid.terrain_nodes = nullptr;
    h->cfg = *cfg;
    h->cfg.knot_z = h->cfg.knot_theta = nullptr;
    h->cfg.qknot_z = h->cfg.qknot_v = nullptr;
    h->user = reinterpret_cast<cudaStream_t>(cuda_stream);
    carve(h, grid, cfg, d_workspace, false);
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    bool terr = false;
    if (grid->terrain_nodes)
        for (long long n = 0; n < (long long)nx * ny; ++n) if (grid->terrain_nodes[n] != 0.0) { terr = true; break; }
    h->geo.terrain = terr ? 1 : 0;
    fill_geo(h);
    // vertical 1D arrays (host, FP64)
    const double *z = grid->z_faces;
    double zt = z[nz];
    std::vector<double> dzeta(nz), zetac(nz), s(nz + 1), sc(nz), ds(nz), dzc(nz + 1, 0.0), d2(nz);
    for (int k = 0; k <= nz; ++k) s[k] = std::pow(1.0 - z[k] / zt, (double)grid->terrain_beta);
    for (int k = 0; k < nz; ++k) {
        dzeta[k] = z[k + 1] - z[k];
        zetac[k] = 0.5 * (z[k] + z[k + 1]);
        sc[k] = 0.5 * (s[k] + s[k + 1]);
        ds[k] = s[k + 1] - s[k];
        double Delta = std::cbrt(grid->dx * grid->dy * dzeta[k]);
        d2[k] = (cfg->Cs * Delta) * (cfg->Cs * Delta);
    }
    for (int k = 1; k < nz; ++k) dzc[k] = zetac[k] - zetac[k - 1];
    std::vector<double> rdzeta(nz), rdzc(nz + 1, 0.0), delta(nz);
    for (int k = 0; k < nz; ++k) rdzeta[k] = 1.0 / dzeta[k];
    for (int k = 0; k < nz; ++k) delta[k] = std::cbrt(grid->dx * grid->dy * dzeta[k]);
    h->ph.ray_zt = zt;
    for (int k = 1; k < nz; ++k) rdzc[k] = 1.0 / dzc[k];
    cudaStream_t st = h->user;
    cudaError_t e;
#define CK(call, where)                                   \
    do {                                                  \
        e = (call);                                       \
        if (e != cudaSuccess) {                           \
            erf_status r = cuda_fail(nullptr, e, where);  \
            delete h;                                     \
            return r;                                     \
        }                                                 \
    } while (0)
    CK(cudaMemcpyAsync(h->dzeta, dzeta.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy dzeta");
    CK(cudaMemcpyAsync(h->zetac, zetac.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy zetac");
    CK(cudaMemcpyAsync(h->s, s.data(), (nz + 1) * sizeof(double), cudaMemcpyHostToDevice, st), "copy s");
    CK(cudaMemcpyAsync(h->sc, sc.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy sc");
    CK(cudaMemcpyAsync(h->ds, ds.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy ds");
    CK(cudaMemcpyAsync(h->dzc, dzc.data(), (nz + 1) * sizeof(double), cudaMemcpyHostToDevice, st), "copy dzc");
    CK(cudaMemcpyAsync(h->delta2, d2.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy delta2");
    CK(cudaMemcpyAsync(h->rdzeta, rdzeta.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy rdzeta");
    CK(cudaMemcpyAsync(h->rdzc, rdzc.data(), (nz + 1) * sizeof(double), cudaMemcpyHostToDevice, st), "copy rdzc");
    CK(cudaMemcpyAsync(h->delta, delta.data(), nz * sizeof(double), cudaMemcpyHostToDevice, st), "copy delta");
    if (cfg->n_knots > 0) {
        CK(cudaMemcpyAsync(h->knz, cfg->knot_z, cfg->n_knots * sizeof(double), cudaMemcpyHostToDevice, st), "copy knots");
        CK(cudaMemcpyAsync(h->knt, cfg->knot_theta, cfg->n_knots * sizeof(double), cudaMemcpyHostToDevice, st), "copy knots");
    }
    long long nxy = (long long)nx * ny;
    if (terr) {
        CK(cudaMemcpyAsync(h->hn, grid->terrain_nodes, nxy * sizeof(double), cudaMemcpyHostToDevice, st), "copy terrain");
    } else {
        CK(cudaMemsetAsync(h->hn, 0, nxy * sizeof(double), st), "zero terrain");
    }
    CK(cudaMemsetAsync(h->kerr, 0, 4 * sizeof(unsigned), st), "zero error word");
    launch_terrain(h->geo, h->hn, h->hc, h->hxf, h->hyf, h->gxh, h->gyh, h->g4xq, h->g4yq, st);
    if (h->geo.terrain && h->rH3)
        launch_terrain_recip(h->geo, h->Hx3, h->Hy3, h->rH3, h->rHx3, h->rHy3, h->rdzw3, h->rdz2, st);
    if (cfg->moist) {
        CK(cudaMemcpyAsync(h->qkz, cfg->qknot_z, cfg->n_qknots * sizeof(double), cudaMemcpyHostToDevice, st), "copy q knots");
        CK(cudaMemcpyAsync(h->qkv, cfg->qknot_v, cfg->n_qknots * sizeof(double), cudaMemcpyHostToDevice, st), "copy q knots");
        CK(cudaMemsetAsync(h->precip, 0, nxy * sizeof(double), st), "zero precipitation");
        for (int q = 0; q < 3; ++q) CK(cudaMemsetAsync(h->rq[q], 0, h->geo.nc * sizeof(double), st), "zero moisture");
    }
    launch_base_state(h->geo, cfg->n_knots, h->knz, h->knt, cfg->theta_s, cfg->brunt_N, cfg->p_s, cfg->gravity,
                      h->rho0, h->th0, h->p0, st, cfg->moist ? cfg->n_qknots : 0, h->qkz, h->qkv, h->qv0);
    std::vector<double> lamx(nx), lamy(ny), twx(nx > 1 ? nx : 2), twy(ny > 1 ? ny : 2);
    if (cfg->anelastic) {
        // eigenvalues of the periodic second differences and the FFT twiddles exp(-2 pi i m / n)
        const double pi_ = 3.141592653589793;
        for (int i = 0; i < nx; ++i) { double sn = std::sin(pi_ * i / nx); lamx[i] = -4.0 / (grid->dx * grid->dx) * sn * sn; }
        for (int j = 0; j < ny; ++j) { double sn = std::sin(pi_ * j / ny); lamy[j] = -4.0 / (grid->dy * grid->dy) * sn * sn; }
        for (int m = 0; m < nx / 2; ++m) { twx[2 * m] = std::cos(2.0 * pi_ * m / nx); twx[2 * m + 1] = -std::sin(2.0 * pi_ * m / nx); }
        for (int m = 0; m < ny / 2; ++m) { twy[2 * m] = std::cos(2.0 * pi_ * m / ny); twy[2 * m + 1] = -std::sin(2.0 * pi_ * m / ny); }
        CK(cudaMemcpyAsync(h->lamx, lamx.data(), nx * sizeof(double), cudaMemcpyHostToDevice, st), "copy eigenvalues");
        CK(cudaMemcpyAsync(h->lamy, lamy.data(), ny * sizeof(double), cudaMemcpyHostToDevice, st), "copy eigenvalues");
        if (nx > 1) CK(cudaMemcpyAsync(h->twx, twx.data(), nx / 2 * sizeof(double2), cudaMemcpyHostToDevice, st), "copy twiddles");
        if (ny > 1) CK(cudaMemcpyAsync(h->twy, twy.data(), ny / 2 * sizeof(double2), cudaMemcpyHostToDevice, st), "copy twiddles");
        CK(cudaMemsetAsync(h->pa, 0, h->geo.nc * sizeof(double), st), "zero pressure");
        if (!anel_fft_setup()) CK(cudaGetLastError(), "FFT shared-memory attribute");
    }
    if (h->mixed) {
        mx_build_base(h->geo, cfg->Cs, grid->dx, grid->dy, cfg->gravity, h->mbase, h->mrt0, st);
        h->mb = mx_base_view(h->mbase, h->mrt0, nz);
        mx_base_scalars(h->mb, h->geo, h->ph);
        h->tma.err = h->kerr;
        h->tma.use = mx_encode_tiles(h) ? 1 : 0;
    }
    CK(cudaGetLastError(), "init kernels");
    CK(cudaStreamSynchronize(st), "init sync");   // host vectors above must outlive the copies
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "create capture stream");
#undef CK
    *out = h;
    return ERF_OK;
}

static CF5 cf(const F5 &f) { return CF5{f.r, f.t, f.u, f.v, f.w}; }
static CF5f cf(const F5f &f) { return CF5f{f.r, f.t, f.u, f.v, f.w}; }

// one RK3 step of the mixed-precision path (flat grids)
// the explicit vertical part runs inside the column sweep once there are enough columns to fill
// the GPU with one thread each.  Measured per step on the convective ABL (160 levels), split vs
// fused: 128^2 columns 7.6 vs 8.5 ms, 256^2 14.3 vs 14.3 ms, 384^2 29.5 vs 24.1 ms, 512^2 49.6 vs
// 43.4 ms; fused also at 1024^2 and 2048^2.
static int fuse_columns(const erf_handle *h) {
    if (h->column_fusion >= 0) return h->column_fusion;
    return h->geo.nxy >= (1LL << 17) ? 1 : 0;
}

static void enqueue_step_mixed(erf_handle *h, cudaStream_t s) {
    const Geo &g = h->geo;
    const Phys &ph = h->ph;
    const erf_config &c = h->cfg;
    mx_wall_bc(g, h->mst.w, s);
    size_t bc = g.nc * sizeof(float), bw = g.nw * sizeof(float);
    // S^n = S^t is written by the first stage's opening pass
    if (h->mtphi) cudaMemcpyAsync(h->msnphi, h->mtphi, bc, cudaMemcpyDeviceToDevice, s);
    const double alpha[3] = {1.0 / 3.0, 0.5, 1.0};
    for (int stage = 0; stage < 3; ++stage) {
        mx_stage_open(g, h->mb, h->msn, cf(h->mst), h->mx, h->mpp, h->mpi, h->mthp, h->mTp, h->mux, h->mvy, h->mwz,
                      h->mmfx, h->mmfy, stage == 0, s);
        ClIn clin{h->cl_w, h->cl_b, h->cl_stats, h->cl_out, h->cl_nfb};
        mx_slow_rhs(g, h->mb, ph, cf(h->mst), h->mpp, h->mthp, h->mux, h->mvy, h->mwz, h->mmfx, h->mmfy, h->mmu,
                    h->mflux, h->mR, s, h->cl_ready ? &clin : nullptr, &h->tma, false);
        int nsub = stage == 0 ? 1 : (stage == 1 ? c.n_substeps / 2 : c.n_substeps);
        double dtau = stage == 0 ? c.dt / 3.0 : c.dt / c.n_substeps;
        mx_tri_build(g, h->mb, ph, h->mst.r, h->mst.t, h->mpi, h->mthp, dtau, h->mtri, s);
        if (h->mtphi) {
            cudaMemsetAsync(h->mms.x, 0, bc, s);
            cudaMemsetAsync(h->mms.y, 0, bc, s);
            cudaMemsetAsync(h->mms.z, 0, bw, s);
        }
        // without a passive scalar (which needs S^t after the substeps) the stage end is folded into
        // the last substep's finishing pass (its float4 form, nx % 4 == 0)
        const bool fold_end = !h->mtphi && g.nx % 4 == 0;
        for (int n = 0; n < nsub; ++n)
            mx_substep(g, h->mb, ph, h->mtri, h->mpi, h->mthp, cf(h->mR), h->mx, h->mTp, h->mdbuf, h->mX0, h->mY0,
                       h->mms, fuse_columns(h), dtau, s, fold_end && n == nsub - 1 ? &h->mst : nullptr);
        // the passive scalar after the substeps, from the stage state S^t (the pressure and flux
        // scratch are free until the next stage begins)
        if (h->mtphi)
            mx_tracer_stage(g, h->mb, ph, h->mst.r, h->mmfx, h->mmfy, h->mst.w, h->msnphi, h->mms, nsub,
                            alpha[stage] * c.dt, h->mpp, h->mflux, h->mtphi, s);
        if (!fold_end) mx_stage_end(g, h->mst, cf(h->mx), s);
    }
}

static AnelWork anel_work(erf_handle *h) {
    // the flux buffer (3 nw doubles) holds the complex field and the mass-density tendency (unused
    // by the anelastic set) the z-solve scratch: both are free during the projection
    return AnelWork{reinterpret_cast<double2 *>(h->flux), h->twx, h->twy, h->lamx, h->lamy, h->R.r, h->pa, h->pan,
                    h->pa1};
}

// one SSP-RK2 step of the anelastic equations (Sec. 3.2), enqueued on stream s:
//   S* = S^n + dt f(S^n), project;  S^{n+1} = S^n + dt/2 (f(S^n) + f(S*)), project
static void enqueue_step_anelastic(erf_handle *h, cudaStream_t s) {
    const Geo &g = h->geo;
    const Phys &ph = h->ph;
    const double dt = h->cfg.dt;
    launch_wall_bc(g, h->st.u, h->st.v, h->st.w, s);
    size_t bc = g.nc * sizeof(double), bw = g.nw * sizeof(double);
    cudaMemcpyAsync(h->sn.t, h->st.t, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.u, h->st.u, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.v, h->st.v, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.w, h->st.w, bw, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->pan, h->pa, bc, cudaMemcpyDeviceToDevice, s);
    Prep pr{h->ux, h->vy, h->wz, h->mfx, h->mfy, h->rom};
    const AnelWork w = anel_work(h);
    for (int stage = 1; stage <= 2; ++stage) {
        launch_anel_begin(g, h->st.t, h->st.r, h->pa, h->pp, h->th, s);
        launch_slow_rhs(g, ph, cf(h->st), h->pp, h->th, pr, h->ux, h->vy, h->wz, h->mfx, h->mfy, h->rom, h->mu,
                        h->flux, h->R, s);
        if (stage == 1) {   // the first stage's tendencies (rho theta, momenta) are kept in x
            cudaMemcpyAsync(h->x.t, h->R.t, bc, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(h->x.u, h->R.u, bc, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(h->x.v, h->R.v, bc, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(h->x.w, h->R.w, bw, cudaMemcpyDeviceToDevice, s);
            launch_anel_stage(g, h->st, cf(h->sn), cf(h->x), cf(h->R), dt, 0.0, s);
        } else {
            launch_anel_stage(g, h->st, cf(h->sn), cf(h->x), cf(h->R), 0.5 * dt, 0.5 * dt, s);
        }
        launch_anel_project(g, w, dt, h->st.u, h->st.v, h->st.w, stage, s);
    }
}

// one RK3 step (Sec. 3.1) with the App. C substeps, enqueued on stream s
static void enqueue_step(erf_handle *h, cudaStream_t s) {
    set_warp_columns(h->warp_columns);
    if (h->mixed) {
        enqueue_step_mixed(h, s);
        return;
    }
    if (h->pa) {
        enqueue_step_anelastic(h, s);
        return;
    }
    const Geo &g = h->geo;
    const Phys &ph = h->ph;
    const erf_config &c = h->cfg;
    launch_wall_bc(g, h->st.u, h->st.v, h->st.w, s);
    size_t bc = g.nc * sizeof(double), bw = g.nw * sizeof(double);
    cudaMemcpyAsync(h->sn.r, h->st.r, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.t, h->st.t, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.u, h->st.u, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.v, h->st.v, bc, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(h->sn.w, h->st.w, bw, cudaMemcpyDeviceToDevice, s);
    if (h->tphi) cudaMemcpyAsync(h->snphi, h->tphi, bc, cudaMemcpyDeviceToDevice, s);
    if (h->tke) cudaMemcpyAsync(h->sntke, h->tke, bc, cudaMemcpyDeviceToDevice, s);
    if (h->rq[0])
        for (int q = 0; q < 3; ++q) cudaMemcpyAsync(h->snq[q], h->rq[q], bc, cudaMemcpyDeviceToDevice, s);
    const double alpha[3] = {1.0 / 3.0, 0.5, 1.0};
    Prep pr{h->ux, h->vy, h->wz, h->mfx, h->mfy, h->rom};
    MoistIO mio{{h->qsrc[0], h->qsrc[1], h->qsrc[2]},
                {h->ref[0], h->ref[1], h->ref[2], h->ref[3], h->ref[4], h->ref[5], h->ref[6], h->ref[7]}};
    const MoistIO *miop = (h->rq[0] || h->ref[0]) ? &mio : nullptr;
    // the moisture scalars after the substeps of a stage: the stage-averaged fluxes, their sources,
    // clipped at zero
    auto moist_stage = [&](int nsub, double adt) {
        if (!h->rq[0]) return;
        for (int q = 0; q < 3; ++q)
            launch_tracer_stage(g, ph, cf(h->st), h->rom, h->snq[q], h->msx, h->msy, h->msz, nsub, adt, h->pp,
                                h->flux, h->rq[q], s, h->qsrc[q], 1);
    };
    for (int stage = 0; stage < 3; ++stage) {
        launch_stage_begin(g, cf(h->sn), cf(h->st), h->x, h->pp, h->pi, h->th, h->Tp, h->Om, s, h->rq[0]);
        launch_slow_rhs(g, ph, cf(h->st), h->pp, h->th, pr, h->ux, h->vy, h->wz, h->mfx, h->mfy, h->rom, h->mu,
                        h->flux, h->R, s, h->tke, h->muh, h->tke_src, miop);
        if (h->msx) {
            cudaMemsetAsync(h->msx, 0, bc, s);
            cudaMemsetAsync(h->msy, 0, bc, s);
            cudaMemsetAsync(h->msz, 0, bw, s);
        }
        if (c.substep_mode == 1) {
            if (h->tphi)
                launch_tracer_stage(g, ph, cf(h->st), h->rom, h->snphi, h->msx, h->msy, h->msz, 1,
                                    alpha[stage] * c.dt, h->pp, h->flux, h->tphi, s);
            if (h->tke)
                launch_tracer_stage(g, ph, cf(h->st), h->rom, h->sntke, h->msx, h->msy, h->msz, 1,
                                    alpha[stage] * c.dt, h->pp, h->flux, h->tke, s, h->tke_src, 1);
            moist_stage(1, alpha[stage] * c.dt);
            launch_stage_nosub(g, h->st, cf(h->sn), cf(h->R), alpha[stage] * c.dt, s);
            launch_wall_bc(g, h->st.u, h->st.v, h->st.w, s);
            continue;
        }
        int nsub = stage == 0 ? 1 : (stage == 1 ? c.n_substeps / 2 : c.n_substeps);
        double dtau = stage == 0 ? c.dt / 3.0 : c.dt / c.n_substeps;
        // the slow-tendency scratch is free once the tendencies exist: the mass-flux arrays take
        // the stage's H theta at faces, the planes of the flux buffer its pressure-gradient
        // factors and w-face theta, the face velocities the substeps' X0, Y0 and metric shift
        double *PX = h->flux, *PY = h->flux + g.nw, *THW = h->flux + 2 * g.nw;
        launch_tri_build(g, ph, h->st.r, h->st.t, h->pi, h->th, dtau, h->tri, h->mfx, h->mfy, PX, PY, THW, s);
        for (int n = 0; n < nsub; ++n)
            launch_substep(g, ph, h->tri, PX, PY, THW, h->mfx, h->mfy, cf(h->R), h->x, h->Om, h->Tp, h->ux, h->vy,
                           h->wz, h->msx, h->msy, h->msz, dtau, s);
        // the passive scalar after the substeps, from the stage state S^t (Sec. 3.1)
        if (h->tphi)
            launch_tracer_stage(g, ph, cf(h->st), h->rom, h->snphi, h->msx, h->msy, h->msz, nsub,
                                alpha[stage] * c.dt, h->pp, h->flux, h->tphi, s);
        if (h->tke)
            launch_tracer_stage(g, ph, cf(h->st), h->rom, h->sntke, h->msx, h->msy, h->msz, nsub,
                                alpha[stage] * c.dt, h->pp, h->flux, h->tke, s, h->tke_src, 1);
        moist_stage(nsub, alpha[stage] * c.dt);
        launch_stage_end(g, h->st, cf(h->x), s);
    }
    // microphysics after the dycore step (time split, Sec. 2.4)
    // (the flux buffer is free once the last stage has ended)
    if (h->rq[0]) launch_kessler(g, c.dt, h->st.t, h->st.r, h->rq[0], h->rq[1], h->rq[2], h->precip, h->flux, s);
}

static erf_status build_graph(erf_handle *h) {
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    enqueue_step(h, h->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "instantiate graph");
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int nk = 0;
    for (auto &n : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(n, &t);
        if (t == cudaGraphNodeTypeKernel) ++nk;
    }
    h->graph = graph;
    h->exec = exec;
    h->kernels_per_step = nk;
    return ERF_OK;
}

extern "C" erf_status erf_rk3_step(erf_handle *h, int32_t nsteps) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (nsteps < 0) return fail(h, ERF_EINVAL, "nsteps < 0");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    if (h->cfg.closure == 3 && !h->cl_ready) return fail(h, ERF_ESTATE, "learned closure weights not set");
    if (!h->exec) {
        erf_status st = build_graph(h);
        if (st != ERF_OK) return st;
    }
    for (int n = 0; n < nsteps; ++n) {
        cudaError_t e = cudaGraphLaunch(h->exec, h->user);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    }
    h->steps_done += nsteps;
    return ERF_OK;
}

namespace {
struct EventSink : ProfSink {
    struct Rec { std::string name; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    void add(const char *name, cudaEvent_t a, cudaEvent_t b) override { recs.push_back({name, a, b}); }
};
}  // namespace

extern "C" erf_status erf_profile_steps(erf_handle *h, int32_t nsteps, erf_kernel_time *out, int32_t max_entries,
                                        int32_t *n_entries) {
    if (!h || !out || !n_entries || max_entries < 1 || nsteps < 1) return fail(h, ERF_EINVAL, "bad profile arguments");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    if (h->cfg.closure == 3 && !h->cl_ready) return fail(h, ERF_ESTATE, "learned closure weights not set");
    EventSink sink;
    set_profiler(&sink);
    for (int n = 0; n < nsteps; ++n) enqueue_step(h, h->user);
    set_profiler(nullptr);
    cudaError_t e = cudaStreamSynchronize(h->user);
    if (e != cudaSuccess) return cuda_fail(h, e, "profile sync");
    h->steps_done += nsteps;
    int n = 0;
    std::vector<std::string> names;
    for (auto &r : sink.recs) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        int idx = -1;
        for (int q = 0; q < n; ++q) if (names[q] == r.name) { idx = q; break; }
        if (idx < 0) {
            if (n >= max_entries) continue;
            idx = n++;
            names.push_back(r.name);
            std::memset(out[idx].name, 0, sizeof(out[idx].name));
            std::strncpy(out[idx].name, r.name.c_str(), sizeof(out[idx].name) - 1);
            out[idx].total_ms = 0.0;
            out[idx].launches = 0;
        }
        out[idx].total_ms += ms;
        out[idx].launches += 1;
    }
    *n_entries = n;
    return ERF_OK;
}

// the prognostic fields in storage order: rho, rho theta, rho u, rho v (nz levels), rho w (nz+1),
// then rho phi when the handle carries the passive scalar
static int state_fields(erf_handle *h, void **ptr, int *levels) {
    const int nz = h->geo.nz;
    int n = 0;
    if (h->mixed) {
        void *f[5] = {h->mst.r, h->mst.t, h->mst.u, h->mst.v, h->mst.w};
        for (int q = 0; q < 5; ++q) { ptr[n] = f[q]; levels[n++] = q == 4 ? nz + 1 : nz; }
        if (h->mtphi) { ptr[n] = h->mtphi; levels[n++] = nz; }
    } else {
        void *f[5] = {h->st.r, h->st.t, h->st.u, h->st.v, h->st.w};
        for (int q = 0; q < 5; ++q) { ptr[n] = f[q]; levels[n++] = q == 4 ? nz + 1 : nz; }
        if (h->tphi) { ptr[n] = h->tphi; levels[n++] = nz; }
        if (h->tke) { ptr[n] = h->tke; levels[n++] = nz; }
        for (int q = 0; q < 3; ++q)
            if (h->rq[q]) { ptr[n] = h->rq[q]; levels[n++] = nz; }
    }
    return n;
}

extern "C" erf_status erf_column_block_bytes(const erf_handle *hc, int32_t ni, int32_t nj, size_t *bytes) {
    erf_handle *h = const_cast<erf_handle *>(hc);
    if (!h || !bytes || ni < 0 || nj < 0) return fail(h, ERF_EINVAL, "bad column-block arguments");
    void *p[12];
    int lv[12];
    int nf = state_fields(h, p, lv);
    size_t words = 0;
    for (int q = 0; q < nf; ++q) words += (size_t)lv[q] * ni * nj;
    *bytes = words * (h->mixed ? sizeof(float) : sizeof(double));
    return ERF_OK;
}

static erf_status column_block(erf_handle *h, int32_t i0, int32_t ni, int32_t j0, int32_t nj, void *buf,
                               int unpack) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    const Geo &g = h->geo;
    if (!buf || ni < 0 || nj < 0 || i0 < 0 || j0 < 0 || (long long)i0 + ni > g.nx || (long long)j0 + nj > g.ny)
        return fail(h, ERF_EINVAL, "column block outside the grid");
    if (unpack == 0 && !h->have_state) return fail(h, ERF_ESTATE, "no state set");
    void *p[12];
    int lv[12];
    int nf = state_fields(h, p, lv);
    const int eb = h->mixed ? (int)sizeof(float) : (int)sizeof(double);
    char *b = reinterpret_cast<char *>(buf);
    for (int q = 0; q < nf; ++q) {
        launch_column_block(p[q], b, eb, g.nx, g.ny, lv[q], i0, ni, j0, nj, unpack, h->user);
        b += (size_t)lv[q] * ni * nj * eb;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, unpack ? "unpack columns" : "pack columns");
    return ERF_OK;
}

extern "C" erf_status erf_pack_columns(erf_handle *h, int32_t i0, int32_t ni, int32_t j0, int32_t nj, void *d_buf) {
    return column_block(h, i0, ni, j0, nj, d_buf, 0);
}

extern "C" erf_status erf_unpack_columns(erf_handle *h, int32_t i0, int32_t ni, int32_t j0, int32_t nj,
                                         const void *d_buf) {
    return column_block(h, i0, ni, j0, nj, const_cast<void *>(d_buf), 1);
}

static erf_status capture_reference(erf_handle *h) {
    if (!h->ref[0]) return ERF_OK;
    const Geo &g = h->geo;
    const double *src[8] = {h->st.r, h->st.t, h->st.u, h->st.v, h->st.w, h->rq[0], h->rq[1], h->rq[2]};
    for (int f = 0; f < 8; ++f) {
        if (!h->ref[f]) continue;
        cudaError_t e = cudaMemcpyAsync(h->ref[f], src[f], (f == 4 ? g.nw : g.nc) * sizeof(double),
                                        cudaMemcpyDeviceToDevice, h->user);
        if (e != cudaSuccess) return cuda_fail(h, e, "capture relaxation reference");
    }
    return ERF_OK;
}

extern "C" erf_status erf_capture_reference(erf_handle *h) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    if (!h->ref[0]) return fail(h, ERF_EUNSUPPORTED, "handle configured without relaxation zones");
    return capture_reference(h);
}

extern "C" erf_status erf_set_initial_moist(erf_handle *h, const double *dtheta, const double *qv, const double *u,
                                            const double *v, const double *w, int32_t is_device) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (!h->rq[0]) return fail(h, ERF_EUNSUPPORTED, "handle configured without moisture");
    const Geo &g = h->geo;
    cudaStream_t s = h->user;
    const double *src[5] = {dtheta, qv, u, v, w};
    double *stage[5] = {h->x.r, h->x.t, h->x.u, h->x.v, h->x.w};   // perturbation arrays as staging
    long long len[5] = {g.nc, g.nc, g.nc, g.nc, g.nw};
    const double *dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int n = 0; n < 5; ++n) {
        if (!src[n]) continue;
        if (is_device) { dev[n] = src[n]; continue; }
        cudaError_t e = cudaMemcpyAsync(stage[n], src[n], len[n] * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy initial field");
        dev[n] = stage[n];
    }
    launch_set_initial_moist(g, dev[0], dev[1], dev[2], dev[3], dev[4], h->st.r, h->st.t, h->st.u, h->st.v, h->st.w,
                             h->rq[0], h->rq[1], h->rq[2], s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_initial_moist kernels");
    h->have_state = true;
    erf_status st = capture_reference(h);
    if (st != ERF_OK) return st;
    if (!is_device) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_initial sync");
    }
    return ERF_OK;
}

extern "C" erf_status erf_set_initial(erf_handle *h, const double *dtheta, const double *u, const double *v,
                                      const double *w, int32_t is_device) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (h->rq[0]) return erf_set_initial_moist(h, dtheta, nullptr, u, v, w, is_device);
    if (h->pa) {
        // anelastic: rho = rho0, rho theta = rho0 theta; the momentum projected once, p' = 0
        const Geo &g = h->geo;
        cudaStream_t s = h->user;
        const double *src[4] = {dtheta, u, v, w};
        double *stage[4] = {h->x.r, h->x.u, h->x.v, h->x.w};
        long long len[4] = {g.nc, g.nc, g.nc, g.nw};
        const double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int n = 0; n < 4; ++n) {
            if (!src[n]) continue;
            if (is_device) { dev[n] = src[n]; continue; }
            cudaError_t e = cudaMemcpyAsync(stage[n], src[n], len[n] * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy initial field");
            dev[n] = stage[n];
        }
        launch_anel_init(g, dev[0], h->st.r, h->st.t, s);
        launch_init_faces(g, dev[1], dev[2], dev[3], h->st.r, h->st.u, h->st.v, h->st.w, s);
        cudaMemsetAsync(h->pa, 0, g.nc * sizeof(double), s);
        launch_anel_project(g, anel_work(h), 1.0, h->st.u, h->st.v, h->st.w, 0, s);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "anelastic initial state");
        h->have_state = true;
        return ERF_OK;
    }
    const Geo &g = h->geo;
    cudaStream_t s = h->user;
    if (h->mixed) {
        // FP64 staging in the (not yet used) LU arrays and solve scratch
        const double *src[4] = {dtheta, u, v, w};
        double *stage[4] = {h->mstage, h->mtri.cp, h->mtri.im, h->mdbuf};
        long long len[4] = {g.nc, g.nc, g.nc, g.nw};
        const double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int n = 0; n < 4; ++n) {
            if (!src[n]) continue;
            if (is_device) { dev[n] = src[n]; continue; }
            cudaError_t e = cudaMemcpyAsync(stage[n], src[n], len[n] * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy initial field");
            dev[n] = stage[n];
        }
        mx_set_initial(g, dev[0], dev[1], dev[2], dev[3], h->mst, s);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && !is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_initial");
        h->have_state = true;
        return ERF_OK;
    }
    const double *src[4] = {dtheta, u, v, w};
    double *stage[4] = {h->x.r, h->x.u, h->x.v, h->x.w};   // perturbation arrays as staging
    long long len[4] = {g.nc, g.nc, g.nc, g.nw};
    const double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int n = 0; n < 4; ++n) {
        if (!src[n]) continue;
        if (is_device) { dev[n] = src[n]; continue; }
        cudaError_t e = cudaMemcpyAsync(stage[n], src[n], len[n] * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "copy initial field");
        dev[n] = stage[n];
    }
    launch_set_initial(g, dev[0], dev[1], dev[2], dev[3], h->st.r, h->st.t, h->st.u, h->st.v, h->st.w, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "set_initial kernels");
    h->have_state = true;
    if (capture_reference(h) != ERF_OK) return ERF_ECUDA;
    if (!is_device) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_initial sync");
    }
    h->have_state = true;
    return ERF_OK;
}

static bool has_tracer(const erf_handle *h) { return h->tphi || h->mtphi; }

static double *field_dev(erf_handle *h, int f, long long &n) {
    const Geo &g = h->geo;
    n = g.nc;
    switch (f) {
    case ERF_RHO: return h->st.r;
    case ERF_RHOTHETA: return h->st.t;
    case ERF_RHOU: return h->st.u;
    case ERF_RHOV: return h->st.v;
    case ERF_RHOW: n = g.nw; return h->st.w;
    case ERF_BASE_RHO: n = g.terrain ? g.nc : g.nz; return h->rho0;
    case ERF_BASE_P: n = g.terrain ? g.nc : g.nz; return h->p0;
    case ERF_BASE_THETA: n = g.terrain ? g.nc : g.nz; return h->th0;
    case ERF_RHOPHI: return h->tphi;
    case ERF_RHOTKE: return h->tke;
    case ERF_RHOQV: return h->rq[0];
    case ERF_RHOQC: return h->rq[1];
    case ERF_RHOQR: return h->rq[2];
    case ERF_PRECIP: n = g.nxy; return h->precip;
    case ERF_BASE_QV: n = g.terrain ? g.nc : g.nz; return h->qv0;
    case ERF_P_ANELASTIC: return h->pa;
    }
    return nullptr;
}

extern "C" erf_status erf_set_state(erf_handle *h, int32_t field, const void *src, int32_t src_is_device,
                                    int32_t src_dtype) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if ((field < ERF_RHO || field > ERF_RHOW) && !(field == ERF_RHOPHI && has_tracer(h)) &&
        !(field == ERF_RHOTKE && h->tke) && !(field >= ERF_RHOQV && field <= ERF_RHOQR && h->rq[0]) &&
        !(field == ERF_P_ANELASTIC && h->pa))
        return fail(h, ERF_EINVAL, "field not settable");
    if (!src) return fail(h, ERF_EINVAL, "src is NULL");
    if (src_dtype != ERF_F64 && src_dtype != ERF_F32) return fail(h, ERF_EINVAL, "bad dtype");
    long long n;
    cudaStream_t s = h->user;
    cudaError_t e;
    if (h->mixed && field == ERF_RHOPHI) {   // rho phi is held whole in FP32
        n = h->geo.nc;
        if (src_dtype == ERF_F32) {
            e = cudaMemcpyAsync(h->mtphi, src, n * sizeof(float),
                                src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        } else {
            const void *d = src;
            e = cudaSuccess;
            if (!src_is_device) {
                e = cudaMemcpyAsync(h->mdbuf, src, n * sizeof(double), cudaMemcpyHostToDevice, s);
                d = h->mdbuf;
            }
            if (e == cudaSuccess) {
                launch_convert(d, h->mtphi, n, 0, s);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess && !src_is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
        return ERF_OK;
    }
    if (h->mixed) {
        float *mf[5] = {h->mst.r, h->mst.t, h->mst.u, h->mst.v, h->mst.w};
        n = field == ERF_RHOW ? h->geo.nw : h->geo.nc;
        const double *d64 = nullptr;
        if (src_dtype == ERF_F64 && src_is_device) d64 = (const double *)src;
        else {
            double *stg = h->mstage;
            if (src_dtype == ERF_F64) {
                e = cudaMemcpyAsync(stg, src, n * sizeof(double), cudaMemcpyHostToDevice, s);
            } else {
                const void *f = src;
                e = cudaSuccess;
                if (!src_is_device) {
                    e = cudaMemcpyAsync(h->mtri.cp, src, n * sizeof(float), cudaMemcpyHostToDevice, s);
                    f = h->mtri.cp;
                }
                if (e == cudaSuccess) launch_convert(f, stg, n, 1, s);
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "copy state");
            d64 = stg;
        }
        mx_from_full(h->geo, d64, mf[field], field, n, s);
        e = cudaGetLastError();
        if (e == cudaSuccess && !src_is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
        h->have_state = true;
        return ERF_OK;
    }
    double *dst = field_dev(h, field, n);
    if (src_dtype == ERF_F64) {
        e = cudaMemcpyAsync(dst, src, n * sizeof(double), src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    } else {
        const void *d = src;
        if (!src_is_device) {
            e = cudaMemcpyAsync(h->x.w, src, n * sizeof(float), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy state");
            d = h->x.w;
        }
        launch_convert(d, dst, n, 1, s);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
    if (!src_is_device) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "set_state sync");
    }
    h->have_state = true;
    return ERF_OK;
}

extern "C" erf_status erf_set_tracer_initial(erf_handle *h, const double *phi0, int32_t is_device) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (!has_tracer(h)) return fail(h, ERF_EUNSUPPORTED, "handle configured without the passive scalar");
    if (!phi0) return fail(h, ERF_EINVAL, "phi0 is NULL");
    const Geo &g = h->geo;
    cudaStream_t s = h->user;
    const double *d = phi0;
    cudaError_t e = cudaSuccess;
    if (!is_device) {
        double *stg = h->mixed ? h->mdbuf : h->snphi;   // FP64 staging of nc values
        e = cudaMemcpyAsync(stg, phi0, g.nc * sizeof(double), cudaMemcpyHostToDevice, s);
        d = stg;
    }
    if (e == cudaSuccess) {
        if (h->mixed) mx_tracer_init(g, h->rho0, h->mst.r, d, h->mtphi, s);
        else launch_tracer_init(g, h->st.r, d, h->tphi, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !is_device) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_tracer_initial");
    return ERF_OK;
}

extern "C" erf_status erf_get_state(erf_handle *h, int32_t field, void *dst, int32_t dst_is_device,
                                    int32_t dst_dtype) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if ((field < ERF_RHO || field > ERF_BASE_THETA) && !(field == ERF_RHOPHI && has_tracer(h)) &&
        !(field == ERF_RHOTKE && h->tke) && !(field >= ERF_RHOQV && field <= ERF_BASE_QV && h->rq[0]) &&
        !(field == ERF_P_ANELASTIC && h->pa))
        return fail(h, ERF_EINVAL, "bad field");
    if (!dst) return fail(h, ERF_EINVAL, "dst is NULL");
    if (dst_dtype != ERF_F64 && dst_dtype != ERF_F32) return fail(h, ERF_EINVAL, "bad dtype");
    long long n;
    cudaStream_t s = h->user;
    cudaError_t e;
    if (h->mixed && field == ERF_RHOPHI) {
        n = h->geo.nc;
        if (dst_dtype == ERF_F32) {
            e = cudaMemcpyAsync(dst, h->mtphi, n * sizeof(float),
                                dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        } else {
            double *stg = dst_is_device ? (double *)dst : h->mdbuf;
            launch_convert(h->mtphi, stg, n, 1, s);
            e = cudaGetLastError();
            if (e == cudaSuccess && !dst_is_device)
                e = cudaMemcpyAsync(dst, stg, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
        return ERF_OK;
    }
    if (h->mixed && field <= ERF_RHOW) {
        const float *mf[5] = {h->mst.r, h->mst.t, h->mst.u, h->mst.v, h->mst.w};
        n = field == ERF_RHOW ? h->geo.nw : h->geo.nc;
        double *stg = (dst_dtype == ERF_F64 && dst_is_device) ? (double *)dst : h->mdbuf;
        mx_to_full(h->geo, mf[field], stg, field, n, s);
        e = cudaGetLastError();
        if (e == cudaSuccess && dst_dtype == ERF_F64 && !dst_is_device)
            e = cudaMemcpyAsync(dst, stg, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && dst_dtype == ERF_F32) {
            void *d = dst_is_device ? dst : (void *)h->mtri.cp;
            launch_convert(stg, d, n, 0, s);
            e = cudaGetLastError();
            if (e == cudaSuccess && !dst_is_device) e = cudaMemcpyAsync(dst, d, n * sizeof(float), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
        return ERF_OK;
    }
    const double *src = field_dev(h, field, n);
    if (dst_dtype == ERF_F64) {
        e = cudaMemcpyAsync(dst, src, n * sizeof(double), dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    } else {
        void *d = dst_is_device ? dst : (void *)h->R.w;   // slow-tendency scratch as staging
        launch_convert(src, d, n, 0, s);
        e = cudaGetLastError();
        if (e == cudaSuccess && !dst_is_device)
            e = cudaMemcpyAsync(dst, d, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
    if (!dst_is_device) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state sync");
    }
    return ERF_OK;
}

extern "C" erf_status erf_diagnostics(erf_handle *h, erf_diag *out) {
    if (!h || !out) return fail(h, ERF_EINVAL, "NULL argument");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    if (h->mixed) mx_diag(h->geo, h->mb, cf(h->mst), h->cfg.dt, h->diag_part, h->diag_out, h->user);
    else launch_diag(h->geo, cf(h->st), h->cfg.dt, h->diag_part, h->diag_out, h->user);
    double v[6];
    unsigned kerr = 0;
    cudaError_t e = cudaMemcpyAsync(v, h->diag_out, sizeof(v), cudaMemcpyDeviceToHost, h->user);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kerr, h->kerr, sizeof(kerr), cudaMemcpyDeviceToHost, h->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->user);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
    if (kerr) return fail(h, ERF_ECUDA, "a kernel's bounded wait for its TMA tile gave up; results are invalid");
    out->mass = v[0];
    out->max_abs_w = v[1];
    out->theta_min = v[2];
    out->theta_max = v[3];
    out->cfl_acoustic = v[4];
    out->nonfinite = v[5] != 0.0;
    out->steps_done = h->steps_done;
    out->kernels_per_step = h->kernels_per_step;
    if (out->nonfinite) return fail(h, ERF_ENONFINITE, "state holds non-finite values");
    return ERF_OK;
}

extern "C" erf_status erf_set_option(erf_handle *h, int32_t option, int64_t value) {
    if (!h) return fail(nullptr, ERF_EINVAL, "NULL handle");
    if (option == ERF_OPT_TMA_STENCILS) {
        h->tma_enabled = value != 0;
        if (h->mixed)
            h->tma.use = (h->tma_enabled && mx_encode_tiles(h)) ? 1 : 0;
    } else if (option == ERF_OPT_COLUMN_FUSION) {
        if (value < -1 || value > 1) return fail(h, ERF_EINVAL, "column fusion must be -1, 0 or 1");
        h->column_fusion = (int)value;
    } else if (option == ERF_OPT_WARP_COLUMNS) {
        if (value < -1 || value > 1) return fail(h, ERF_EINVAL, "warp columns must be -1, 0 or 1");
        h->warp_columns = (int)value;
    } else {
        return fail(h, ERF_EINVAL, "unknown option");
    }
    // the captured step graph holds the previous choice
    if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    return ERF_OK;
}
extern "C" erf_status erf_selftest_wait_timeout(int32_t max_polls, unsigned *d_flag, void *cuda_stream,
                                                int32_t *timed_out) {
    if (!d_flag || !timed_out || max_polls < 1) return fail(nullptr, ERF_EINVAL, "bad self-test arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        selftest_wait_timeout(max_polls, d_flag, s);
        e = cudaGetLastError();
    }
    unsigned f = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f, d_flag, sizeof(f), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "wait self-test");
    *timed_out = f ? 1 : 0;
    return ERF_OK;
}
extern "C" erf_status erf_selftest_tensor_cores(int32_t *d_words, void *cuda_stream, int32_t *mismatches,
                                                 int32_t *timed_out) {
    if (!d_words || !mismatches || !timed_out) return fail(nullptr, ERF_EINVAL, "bad self-test arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(d_words, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        selftest_tensor_cores(d_words, reinterpret_cast<unsigned *>(d_words + 1), s);
        e = cudaGetLastError();
    }
    int32_t w[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, d_words, sizeof(w), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tensor-core self-test");
    *mismatches = w[0];
    *timed_out = w[1] ? 1 : 0;
    return ERF_OK;
}
extern "C" erf_status erf_get_option(erf_handle *h, int32_t option, int64_t *value) {
    if (!h || !value) return fail(h, ERF_EINVAL, "NULL argument");
    if (option == ERF_OPT_TMA_STENCILS) *value = (h->mixed && h->tma.use) ? 1 : 0;
    else if (option == ERF_OPT_COLUMN_FUSION) *value = (h->mixed && fuse_columns(h)) ? 1 : 0;
    else if (option == ERF_OPT_WARP_COLUMNS)
        *value = (!h->mixed && h->geo.nz <= 256 &&
                  (h->warp_columns >= 0 ? h->warp_columns == 1 : h->geo.nxy < (1LL << 15))) ? 1 : 0;
    else return fail(h, ERF_EINVAL, "unknown option");
    return ERF_OK;
}

// ---------------------------------------------------------------- learned closure entry points
extern "C" erf_status erf_set_closure_weights(erf_handle *h, const void *blob, size_t bytes) {
    if (!h || !blob) return fail(h, ERF_EINVAL, "NULL argument");
    if (h->cfg.closure != 3 || !h->cl_w) return fail(h, ERF_EINVAL, "handle was not configured with the learned closure");
    if (bytes != 8 + sizeof(float) * CL_BLOB_FLOATS) return fail(h, ERF_EINVAL, "closure blob has the wrong size");
    unsigned magic;
    std::memcpy(&magic, blob, 4);
    if (magic != CL_MAGIC) return fail(h, ERF_EINVAL, "closure blob has the wrong magic");
    cudaStream_t s = h->user;
    cudaError_t e = cudaMemcpyAsync(h->cl_blob, (const char *)blob + 8, sizeof(float) * CL_BLOB_FLOATS,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy closure blob");
    cl_prepare(h->cl_blob, h->cl_w, h->cl_b, h->cl_stats, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "prepare closure weights");
    h->cl_ready = true;
    // the captured step graph (if any) was built without the closure pointers being live
    if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    return ERF_OK;
}

// EOS + face velocities of the current state (mixed path) into the stage scratch
static void mx_current_fields(erf_handle *h, cudaStream_t s) {
    mx_stage_begin(h->geo, h->mb, cf(h->mst), cf(h->mst), h->mx, h->mpp, h->mpi, h->mthp, h->mTp, s);
    mx_slow_prep_only(h->geo, h->mb, cf(h->mst), h->mux, h->mvy, h->mwz, h->mmfx, h->mmfy, s);
}

extern "C" erf_status erf_closure_features(erf_handle *h, float *d_out) {
    if (!h || !d_out) return fail(h, ERF_EINVAL, "NULL argument");
    if (!h->mixed) return fail(h, ERF_EUNSUPPORTED, "closure features are built on the mixed-precision path");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    mx_current_fields(h, h->user);
    cl_features_launch(h->geo, h->mb, h->cfg.gravity, h->mux, h->mvy, h->mwz, h->mthp, d_out, h->user);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ERF_OK : cuda_fail(h, e, "closure features");
}

extern "C" erf_status erf_closure_fields(erf_handle *h, float *d_out9, uint32_t *n_fallback) {
    if (!h || !d_out9) return fail(h, ERF_EINVAL, "NULL argument");
    if (!h->cl_ready) return fail(h, ERF_ESTATE, "learned closure weights not set");
    if (!h->have_state) return fail(h, ERF_ESTATE, "no state set");
    cudaStream_t s = h->user;
    mx_current_fields(h, s);
    cudaMemsetAsync(h->cl_nfb, 0, sizeof(unsigned), s);
    cl_infer(h->geo, h->mb, h->ph, h->cl_w, h->cl_b, h->cl_stats, h->mux, h->mvy, h->mwz, h->mthp, h->mst.r, d_out9,
             h->cl_nfb, h->kerr, s);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && n_fallback) {
        e = cudaMemcpyAsync(n_fallback, h->cl_nfb, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e == cudaSuccess ? ERF_OK : cuda_fail(h, e, "closure fields");
}

extern "C" erf_status erf_filter_state(erf_handle *h, int32_t r, double *d_rho, double *d_rhotheta, double *d_rhou,
                                       double *d_rhov, double *d_rhow, float *d_targets) {
    if (!h || !d_rho || !d_rhotheta || !d_rhou || !d_rhov || !d_rhow || !d_targets) return fail(h, ERF_EINVAL, "NULL argument");
    if (!h->mixed) return fail(h, ERF_EUNSUPPORTED, "the filter reads the mixed-precision state");
    const Geo &g = h->geo;
    if (r < 1 || g.nx % r || g.ny % r || g.nz % r) return fail(h, ERF_EINVAL, "grid not divisible by the filter ratio");
    for (int k = 0; k < g.nz; ++k) (void)k;
    cl_filter_launch(g, h->mb, cf(h->mst), r, d_rho, d_rhotheta, d_rhou, d_rhov, d_rhow, d_targets, h->user);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ERF_OK : cuda_fail(h, e, "filter");
}

extern "C" const char *erf_last_error(const erf_handle *h) {
    return h ? h->err.c_str() : g_init_error.c_str();
}

extern "C" void erf_destroy(erf_handle *h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}
