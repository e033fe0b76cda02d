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
                       double p_s, double grav, double *rho0, double *th0, double *p0, cudaStream_t s);
void launch_set_initial(const Geo &g, const double *dth, const double *u, const double *v, const double *w,
                        double *rho, double *rt, double *ru, double *rv, double *rw, cudaStream_t s);
void launch_wall_bc(const Geo &g, const double *ru, const double *rv, double *rw, cudaStream_t s);
void launch_stage_begin(const Geo &g, CF5 sn, CF5 st, F5 x, double *pp, double *pi, double *th, double *Tp,
                        double *Om, cudaStream_t s);
void launch_slow_rhs(const Geo &g, const Phys &ph, CF5 st, double *pp, const double *th, Prep pr,
                     double *ux, double *vy, double *wz, double *mfx, double *mfy, double *rom, double *mu,
                     double *flux, F5 R, cudaStream_t s, const double *rtke = nullptr, double *muh = nullptr,
                     double *tke_src = nullptr);
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

// receives (kernel name, start event, stop event) for every launch while profiling is on
struct ProfSink {
    virtual void add(const char *name, cudaEvent_t start, cudaEvent_t stop) = 0;
    virtual ~ProfSink() {}
};
void set_profiler(ProfSink *p);
ProfSink *current_profiler();

}  // namespace erfk
