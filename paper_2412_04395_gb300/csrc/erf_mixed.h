// Mixed-precision (FP32 perturbation) path: data structures and launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "erf_dev.cuh"
#include "erf_launch.h"

namespace erfk {

// FP32 prognostic perturbation fields: drho, d(rho theta), rho u, rho v, rho w
struct F5f {
    float *r, *t, *u, *v, *w;
};
struct CF5f {
    const float *r, *t, *u, *v, *w;
};

// per-level base-state tables of a flat grid (FP32 copies for the FP32 stencils, FP64 where a
// value enters a difference or the tridiagonal)
struct MxBase {
    const float *rho0f, *th0f, *p0f, *pi0f, *rrt0f;   // [nz]; rrt0f = 1/(rho0 theta0)
    const float *rhowf;                               // [nz+1] face-averaged rho0
    const float *dzf, *rdzf, *rdzcf, *delta2f;        // [nz], [nz], [nz+1], [nz]
    const double *rt0;                                // [nz] rho0 theta0 (FP64)
    const float *dth0t;                               // [nz][7]: theta0(k+o) - theta0(k), o = -3..3, formed in FP64
    const float *gth0f;                               // [nz] g / theta0
    const float *r2dzf;                               // [nz] 1/(zc(ku) - zc(kl)), kl = max(k-1,0), ku = min(k+1,nz-1)
    // FP32 copies of the scalar parameters, converted once on the host: a double-to-float
    // conversion per thread would occupy GB300's FP64 pipe (1/64 of the FP32 rate)
    float rdx, rdy, grav, f_cor, u_g, v_g, nu, z0, Qs, rPr, b1, b2, bd;
};
// fills the scalar members from the grid and the physics parameters (host)
inline void mx_base_scalars(MxBase &mb, const Geo &g, const Phys &ph) {
    mb.rdx = (float)g.rdx; mb.rdy = (float)g.rdy; mb.grav = (float)ph.g; mb.f_cor = (float)ph.f_cor;
    mb.u_g = (float)ph.u_g; mb.v_g = (float)ph.v_g; mb.nu = (float)ph.nu; mb.z0 = (float)ph.z0; mb.Qs = (float)ph.Qs;
    mb.rPr = (float)(1.0 / ph.Pr_t); mb.b1 = (float)(0.5 * (1.0 - ph.beta_s)); mb.b2 = (float)(0.5 * (1.0 + ph.beta_s));
    mb.bd = (float)ph.beta_d;
}
// theta0(ka) - theta0(kb) for |ka - kb| <= 3 (ka reflected at the walls)
__device__ __forceinline__ float mx_dth0(const MxBase &mb, int ka, int kb) { return mb.dth0t[kb * 7 + (ka - kb) + 3]; }

// stage LU factors of the vertical system in FP64 and its right-hand-side coefficients in FP32
// a (the sub-diagonal) is formed in FP32 from the FP32 stage fields, so it is stored in FP32 with
// no loss; the elimination reads it as the exact FP64 value
struct TriM {
    float *a;
    double *cp, *im;
    float *P, *Q;
};

// profiling hook shared with the FP64 launchers
ProfSink *current_profiler();
template <class F>
inline void mx_launch(const char *name, cudaStream_t s, F &&launch) {
    ProfSink *p = current_profiler();
    cudaEvent_t a = nullptr, b = nullptr;
    if (p) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    launch();
    if (p) {
        cudaEventRecord(b, s);
        p->add(name, a, b);
    }
}

// learned closure inputs of a slow-tendency pass
struct ClIn {
    const void *w;        // BF16 weights (padded layout)
    const float *b, *stats;
    float *out;           // 9 planes of nc floats
    unsigned *nfb;        // fallback counter (may be null)
};
void cl_prepare(const float *d_blob, void *w_bf16, float *b, float *stats, cudaStream_t s);
void cl_infer(const Geo &g, const MxBase &mb, const Phys &ph, const void *w_bf16, const float *b,
              const float *stats, const float *ux, const float *vy, const float *wz, const float *thp,
              const float *dr, float *out, unsigned *nfb, unsigned *err, cudaStream_t s);
void selftest_tensor_cores(int *mism, unsigned *flag, cudaStream_t s);
void cl_features_launch(const Geo &g, const MxBase &mb, double grav, const float *ux, const float *vy,
                        const float *wz, const float *thp, float *out, cudaStream_t s);
void cl_filter_launch(const Geo &g, const MxBase &mb, CF5f st, int r, double *cr, double *crt, double *cru,
                      double *crv, double *crw, float *targets, cudaStream_t s);

void launch_diag_final(const double *part, int nparts, double dt, double *out, cudaStream_t s);
void mx_build_base(const Geo &g, double Cs, double dx, double dy, double grav, float *f32, double *rt0, cudaStream_t s);
void mx_set_initial(const Geo &g, const double *dth, const double *u, const double *v, const double *w, F5f st,
                    cudaStream_t s);
void mx_from_full(const Geo &g, const double *src, float *dst, int field, long long n, cudaStream_t s);
void mx_to_full(const Geo &g, const float *src, double *dst, int field, long long n, cudaStream_t s);
void mx_wall_bc(const Geo &g, float *rw, cudaStream_t s);
void mx_stage_begin(const Geo &g, const MxBase &mb, CF5f sn, CF5f st, F5f x, float *pp, float *pi, float *thp,
                    float *Tp, cudaStream_t s);
// TMA tile maps of the stencil fields (use = 0: the plain-load kernels) and the device word a
// kernel sets when a bounded wait gives up
struct MxTma {
    CUtensorMap thp, ux, vy, wz;
    int use;
    unsigned *err;
};
bool mx_encode_cell_tile_map(CUtensorMap *map, const float *base, const Geo &g, int nlev);
void selftest_wait_timeout(int max_polls, unsigned *flag, cudaStream_t s);
void mx_slow_rhs(const Geo &g, const MxBase &mb, const Phys &ph, CF5f st, const float *pp, const float *thp,
                 float *ux, float *vy, float *wz, float *mfx, float *mfy, float *mu, float *flux, F5f R, cudaStream_t s,
                 const ClIn *cl, const MxTma *tma, bool prep = true);
// the stage's opening pass: EOS quantities, X'' and the face velocities / mass fluxes in one
// kernel (first: the step's first stage, which also writes the S^n copy)
void mx_stage_open(const Geo &g, const MxBase &mb, F5f sn, CF5f st, F5f x, float *pp, float *pi, float *thp,
                   float *Tp, float *ux, float *vy, float *wz, float *mfx, float *mfy, bool first, cudaStream_t s);
void mx_slow_prep_only(const Geo &g, const MxBase &mb, CF5f st, float *ux, float *vy, float *wz, float *mfx,
                       float *mfy, cudaStream_t s);
void mx_tri_build(const Geo &g, const MxBase &mb, const Phys &ph, const float *dr, const float *dT, const float *pi,
                  const float *thp, double dtau, TriM tr, cudaStream_t s);
// passive-scalar sums of the substeps' perturbation momenta U'', V'' and vertical flux
// b1 Omega''^tau + b2 Omega''^(tau+dtau) (all null without the scalar)
struct TrSum {
    float *x, *y, *z;
};
// one acoustic substep; fuse_columns = 1 runs the explicit vertical part inside the column
// sweep (k_mx_sub_vert), 0 as its own per-cell kernel before the sweep
void mx_substep(const Geo &g, const MxBase &mb, const Phys &ph, TriM tr, const float *pi, const float *thp, CF5f R,
                F5f x, float *Tt, double *dbuf, float *X0, float *Y0, TrSum ms, int fuse_columns, double dtau,
                cudaStream_t s, const F5f *stage_end = nullptr);
void mx_stage_end(const Geo &g, F5f st, CF5f x, cudaStream_t s);
// rho phi^(s) from S^n's rho phi and the stage's averaged mass fluxes (phi and flux are scratch)
void mx_tracer_stage(const Geo &g, const MxBase &mb, const Phys &ph, const float *dr, const float *mfx,
                     const float *mfy, const float *rw, const float *snphi, TrSum ms, int nsub, double adt,
                     float *phi, float *flux, float *rphi, cudaStream_t s);
void mx_tracer_init(const Geo &g, const double *rho0, const float *dr, const double *phi0, float *rphi,
                    cudaStream_t s);
void mx_diag(const Geo &g, const MxBase &mb, CF5f st, double dt, double *part, double *out, cudaStream_t s);

// layout of the FP32 base table block built by mx_build_base (offsets in floats)
// tables in order: rho0, theta0, p0, pi0, 1/(rho0 theta0), rho0 at w-faces, dz, 1/dz, 1/dzc, delta^2
// (nz+1 each), the theta0 differences (7 nz), g/theta0 and the centred 1/dz (nz+1 each)
inline int mx_base_floats(int nz) { return 12 * (nz + 1) + 7 * nz; }
inline MxBase mx_base_view(const float *f32, const double *rt0, int nz) {
    int L = nz + 1;
    const float *tail = f32 + 10 * L + 7 * nz;
    return MxBase{f32, f32 + L, f32 + 2 * L, f32 + 3 * L, f32 + 4 * L, f32 + 5 * L,
                  f32 + 6 * L, f32 + 7 * L, f32 + 8 * L, f32 + 9 * L, rt0, f32 + 10 * L, tail, tail + L,
                  0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
}

}  // namespace erfk
