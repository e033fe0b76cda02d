// Kernel launchers of the dycore library (host-callable, stream-ordered, capturable).
#pragma once
#include <cuda_runtime.h>

#include "erf_dev.cuh"

namespace erfk {

void launch_terrain(const Geo &g, const double *hn, double *hc, double *hxf, double *hyf, double *gxh,
                    double *gyh, double *g4xq, double *g4yq, cudaStream_t s);
void launch_terrain_recip(const Geo &g, double *Hx3, double *Hy3, double *rH3, double *rHx3, double *rHy3,
                          double *rdzw3, double *rdz2, cudaStream_t s);
void launch_base_state(const Geo &g, int n_knots, const double *kz, const double *kt, double theta_s, double N,
                       double p_s, double grav, double *rho0, double *th0, double *p0, cudaStream_t s,
                       int n_qknots = 0, const double *qz = nullptr, const double *qk = nullptr, double *qv0 = nullptr);
void launch_set_initial_moist(const Geo &g, const double *dth, const double *qv, const double *u, const double *v,
                              const double *w, double *rho, double *rt, double *ru, double *rv, double *rw,
                              double *rqv, double *rqc, double *rqr, cudaStream_t s);
// fscratch: nc doubles for the rain-fall fluxes
void launch_kessler(const Geo &g, double dt, double *rt, const double *rho, double *rqv, double *rqc, double *rqr,
                    double *precip, double *fscratch, cudaStream_t s);
// moisture sources of the slow pass (diffusion, relaxation) and the relaxation reference state:
// ref[0..4] = rho, rho theta, rho u, rho v, rho w; ref[5..7] = rho q_v, q_c, q_r (ref[0] null: no
// relaxation zones); src[0..2] receive the moisture sources
struct MoistIO {
    double *src[3];
    const double *ref[8];
};
void launch_set_initial(const Geo &g, const double *dth, const double *u, const double *v, const double *w,
                        double *rho, double *rt, double *ru, double *rv, double *rw, cudaStream_t s);
void launch_wall_bc(const Geo &g, const double *ru, const double *rv, double *rw, cudaStream_t s);
// face momenta u, v, w times the face-averaged density (NULL velocity = 0), then the wall rows
void launch_init_faces(const Geo &g, const double *u, const double *v, const double *w, const double *rho,
                       double *ru, double *rv, double *rw, cudaStream_t s);
void launch_stage_begin(const Geo &g, CF5 sn, CF5 st, F5 x, double *pp, double *pi, double *th, double *Tp,
                        double *Om, cudaStream_t s, const double *rqv = nullptr);
void launch_slow_rhs(const Geo &g, const Phys &ph, CF5 st, double *pp, const double *th, Prep pr,
                     double *ux, double *vy, double *wz, double *mfx, double *mfy, double *rom, double *mu,
                     double *flux, F5 R, cudaStream_t s, const double *rtke = nullptr, double *muh = nullptr,
                     double *tke_src = nullptr, const MoistIO *mio = nullptr);
void launch_tri_build(const Geo &g, const Phys &ph, const double *rho, const double *rt, const double *pi,
                      const double *th, double dtau, Tri tr, double *TX, double *TY, double *PX, double *PY,
                      double *THW, cudaStream_t s);
void launch_substep(const Geo &g, const Phys &ph, Tri tr, const double *PX, const double *PY, const double *thw,
                    const double *TX, const double *TY, CF5 R, F5 x, double *Om, double *Tp, double *X0, double *Y0,
                    double *Ash, double *msx, double *msy, double *msz, double dtau, cudaStream_t s);
void launch_tracer_stage(const Geo &g, const Phys &ph, CF5 st, const double *rom, const double *snphi,
                         const double *msx, const double *msy, const double *msz, int nsub, double adt,
                         double *phi, double *flux, double *rphi, cudaStream_t s, const double *src = nullptr,
                         int clip = 0);
void launch_tracer_init(const Geo &g, const double *rho, const double *phi0, double *rphi, cudaStream_t s);
void launch_stage_end(const Geo &g, F5 st, CF5 x, cudaStream_t s);
void launch_stage_nosub(const Geo &g, F5 st, CF5 sn, CF5 R, double adt, cudaStream_t s);
void launch_diag(const Geo &g, CF5 st, double dt, double *part, double *out, cudaStream_t s);
void launch_convert(const void *src, void *dst, long long n, int to_f64, cudaStream_t s);
// copies the columns [i0, i0+ni) x [j0, j0+nj) of one field (levels x ny x nx, elem_bytes 8 or 4)
// to (unpack = 0) or from (unpack = 1) a packed buffer [levels][nj][ni]
void launch_column_block(void *field, void *buf, int elem_bytes, int nx, int ny, int levels, int i0, int ni,
                         int j0, int nj, int unpack, cudaStream_t s);

constexpr int DIAG_PARTS = 512;
// mode of the one-warp-per-column kernels for the launches that follow (-1 by column count)
void set_warp_columns(int mode);

// receives (kernel name, start event, stop event) for every launch while profiling is on
struct ProfSink {
    virtual void add(const char *name, cudaEvent_t start, cudaEvent_t stop) = 0;
    virtual ~ProfSink() {}
};
void set_profiler(ProfSink *p);
ProfSink *current_profiler();
// an event pair around the launches of its scope while profiling is on
struct ProfLaunch {
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfLaunch(const char *n, cudaStream_t st) : s(st), name(n) {
        if (current_profiler()) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
        }
    }
    ~ProfLaunch() {
        if (ProfSink *p = current_profiler()) {
            cudaEventRecord(b, s);
            p->add(name, a, b);
        }
    }
};

// anelastic projection (Sec. 3.2): complex work field cw (nc), twiddles exp(-2 pi i m / n) of the
// x and y transforms (n/2 each), the eigenvalues lamx[nx], lamy[ny] of the periodic second
// differences, nc scratch values cp of the z solves, the pressure p' (pa), its value at the step
// start (pan) and after the first stage (pa1)
struct AnelWork {
    double2 *cw;
    const double2 *twx, *twy;
    const double *lamx, *lamy;
    double *cp, *pa, *pan, *pa1;
};
void launch_anel_begin(const Geo &g, const double *rt, const double *rho, const double *pa, double *pp, double *th,
                       cudaStream_t s);
void launch_anel_stage(const Geo &g, F5 st, CF5 sn, CF5 R1, CF5 R, double a, double b, cudaStream_t s);
void launch_anel_init(const Geo &g, const double *dth, double *rho, double *rt, cudaStream_t s);
// stage 0: projection only (the initial state); 1, 2: the SSP-RK2 stages with their pressure update
void launch_anel_project(const Geo &g, const AnelWork &w, double dt, double *mu, double *mv, double *mw, int stage,
                         cudaStream_t s);
bool anel_fft_setup();

}  // namespace erfk
