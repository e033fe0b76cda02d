/*
 * erf.h - C ABI of the GB300 (sm_103a) implementation of one RK3 step of ERF's compressible
 * dynamical core (Lattanzi et al., "ERF: Energy Research and Forecasting Model", arXiv 2412.04395).
 *
 * The library advances the dry compressible equations (Sec. 2.1, Eqs. con, mom, theta with the
 * EOS p = P00 (R_d rho theta / P00)^gamma, p' = p - p0, B = -(rho - rho0) g) with the low-storage
 * RK3 of Sec. 3.1 and, inside each stage, the semi-implicit acoustic substeps of App. C (one
 * vertical tridiagonal solve per column).  The grid is the Arakawa C-grid of Sec. 3.4 with the
 * terrain-following height coordinate z = zeta + (1 - zeta/z_t)^beta h(x,y) and the discrete
 * metric terms of App. B.  Lateral boundaries are periodic; bottom and top are walls (Omega = 0)
 * with slip or MOST surface fluxes at the bottom.
 *
 * Plain C types only.  Memory model:
 *   - The caller owns one device workspace (size from erf_workspace_bytes) and the CUDA stream.
 *     The library never calls cudaMalloc; all state, base state, metrics and scratch live in that
 *     workspace.  The workspace must stay valid until erf_destroy.
 *   - The library owns the host handle (erf_destroy frees it) and a private capture stream.
 *   - Every call is asynchronous on the caller's stream except erf_diagnostics and the host-side
 *     variants of erf_get_state, which synchronise the stream.
 * Errors: every entry point returns erf_status; nothing throws or exits.  erf_last_error gives a
 * message for the last failed call on a handle.
 *
 * Field layout (C order [k][j][i], i fastest, periodic faces stored once):
 *   cell fields  (rho, rho*theta)       nz * ny * nx, cell (i,j,k) centred at ((i+1/2)dx, (j+1/2)dy)
 *   rho*u  on x-faces                   nz * ny * nx, face i at x = i dx (left face of cell i)
 *   rho*v  on y-faces                   nz * ny * nx, face j at y = j dy
 *   rho*w  on w-faces                   (nz+1) * ny * nx, face k = bottom face of cell k
 * The boundary rows k = 0 and k = nz of rho*w are derived (Omega = 0 on the walls) and are
 * recomputed at the start of every step.
 */
#ifndef ERF_GB300_H
#define ERF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct erf_handle erf_handle;

typedef enum {
    ERF_OK = 0,
    ERF_EINVAL = -1,        /* invalid argument (sizes, enums, NULL pointers) */
    ERF_ENOSPACE = -2,      /* workspace smaller than erf_workspace_bytes */
    ERF_ECUDA = -3,         /* a CUDA runtime call failed; see erf_last_error */
    ERF_ENONFINITE = -4,    /* the state holds a NaN/Inf (sticky until the state is set again) */
    ERF_ESTATE = -5,        /* step requested before any state was set */
    ERF_EUNSUPPORTED = -6   /* valid but unsupported combination (e.g. SGS over terrain) */
} erf_status;

typedef enum {
    ERF_RHO = 0, ERF_RHOTHETA = 1, ERF_RHOU = 2, ERF_RHOV = 3, ERF_RHOW = 4,
    ERF_BASE_RHO = 5, ERF_BASE_P = 6, ERF_BASE_THETA = 7,    /* base state: get only */
    ERF_RHOPHI = 8,                 /* passive scalar rho phi at cells (config tracer = 1) */
    ERF_RHOTKE = 9,                 /* rho e, the SGS kinetic energy of the Deardorff closure */
    ERF_RHOQV = 10, ERF_RHOQC = 11, ERF_RHOQR = 12,   /* rho q_v, rho q_c, rho q_r (moist handles) */
    ERF_PRECIP = 13,                /* accumulated surface precipitation [m of water], ny*nx, get only */
    ERF_BASE_QV = 14,               /* base-state water vapour q_v0, get only (layout of the base state) */
    ERF_P_ANELASTIC = 15            /* the anelastic pressure perturbation p' at cells (anelastic handles) */
} erf_field;

typedef enum { ERF_F64 = 0, ERF_F32 = 1 } erf_dtype;
typedef enum { ERF_PREC_FP64 = 0, ERF_PREC_MIXED32 = 1 } erf_precision;
typedef enum { ERF_CLOSURE_NONE = 0, ERF_CLOSURE_CONST_NU = 1, ERF_CLOSURE_SMAGORINSKY = 2,
               ERF_CLOSURE_LEARNED = 3 /* mixed precision only */,
               ERF_CLOSURE_DEARDORFF = 4 /* FP64 path, flat grids */ } erf_closure;
typedef enum { ERF_SCAL_WENO5_JS = 0, ERF_SCAL_WENO5_Z = 1, ERF_SCAL_UPWIND3 = 3 } erf_scalar_scheme;
typedef enum { ERF_SURFACE_SLIP = 0, ERF_SURFACE_MOST = 1 } erf_surface;

/* Grid (Sec. 3.4, App. A/B).  Host pointers, read during erf_init_grid only. */
typedef struct {
    int32_t nx, ny, nz;             /* cells; nx >= 1, 1 <= ny <= 65535, 1 <= nz <= ERF_NZ_MAX,
                                       nx*ny*(nz+1) < 2^31 (else ERF_EINVAL) */
    double dx, dy;                  /* uniform horizontal spacing [m] */
    const double *z_faces;          /* nz+1 flat-column face heights zeta_k, increasing, z_faces[0] = 0 */
    const double *terrain_nodes;    /* ny*nx terrain heights h at nodes (i dx, j dy), or NULL = flat */
    int32_t terrain_beta;           /* canonical smoothing exponent: 1 = BTF, 3 = Sullivan */
} erf_grid_desc;

#define ERF_NZ_MAX 512

/* Run configuration.  Where the paper is silent, the library takes the readings stated with each
 * field and entry point below; defaults are those of the paper where it gives them. */
typedef struct {
    double dt;                      /* RK3 step [s] */
    int32_t n_substeps;             /* acoustic substeps per dt (even); stage 1 uses 1 of dt/3 (Sec. 3.3) */
    int32_t substep_mode;           /* 0 = semi-implicit substeps (App. C), 1 = none (plain RK3, Sec. 3.1) */
    double beta_s;                  /* off-centering, beta_1 = (1-beta_s)/2, beta_2 = (1+beta_s)/2 (App. C) */
    double beta_d;                  /* divergence damping of the forward-predicted pressure (Sec. 3.1) */
    int32_t scal_adv;               /* erf_scalar_scheme (Sec. 3.6): WENO5-JS, WENO5-Z or the linear
                                       third-order upwind interpolant */
    int32_t closure;                /* erf_closure (Sec. 2.3).  ERF_CLOSURE_DEARDORFF: the 1.5-order
                                       TKE model of Deardorff (1980) with the coefficients of Moeng
                                       (1984): l = Delta = (dx dy dz)^(1/3), or 0.76 sqrt(e)/N when
                                       shorter in stable air; mu = rho 0.1 l sqrt(e) in the stress,
                                       rho K_h = (1 + 2 l/Delta) mu for the heat flux; rho e is a
                                       transported scalar (the stage-averaged fluxes of Sec. 3.1) with
                                       the source rho (P - K_h N^2 - C_eps e^(3/2)/l) + div(2 mu grad e),
                                       P the energy the stress takes from the resolved flow, C_eps =
                                       0.19 + 0.51 l/Delta, clipped at rho e >= 0.  Initial rho e is set
                                       with erf_set_state(ERF_RHOTKE) (zero otherwise). */
    double Cs, Pr_t, nu;            /* Smagorinsky constant, turbulent Prandtl number, constant nu [m^2/s] */
    int32_t precision;              /* erf_precision */
    double gravity;                 /* g [m/s^2] (0 allowed) */
    double f_cor, u_g, v_g;         /* f-plane Coriolis [1/s] and geostrophic wind [m/s] (Sec. 3.7) */
    int32_t surface;                /* erf_surface (Sec. 3.8) */
    double z0, sfc_theta_flux;      /* MOST roughness [m], surface kinematic heat flux [K m/s] */
    double theta_s, brunt_N, p_s;   /* base state theta0 = theta_s exp(N^2 z/g), surface pressure at z = 0 */
    int32_t n_knots;                /* > 0: theta0 from a piecewise-linear sounding instead */
    const double *knot_z, *knot_theta;   /* host, n_knots each, read during erf_init_grid only */
    int32_t tracer;                 /* 1 = advance a passive scalar rho phi (Sec. 3.1: after the
                                       substeps of each stage, with the stage-averaged momenta that
                                       advanced rho; FP64, or whole FP32 values on the mixed path);
                                       0 = none */
    int32_t mom_adv;                /* momentum interpolant order (Sec. 3.6): 5 (or 0) upwind-5,
                                       3 upwind-3 (the paper's scaling workload, Sec. 5.2) */
    double ray_tau, ray_zd;         /* Rayleigh damping (Sec. 3.7, App. D; FP64 path): rate [1/s] at
                                       the domain top, ramped by sin^2 from 0 at height ray_zd [m];
                                       each damped quantity relaxes at its own physical height,
                                       -tau(z) rho (phi - phi_ref), toward u_g, v_g, 0 and the base
                                       theta0.  ray_tau = 0 or ray_fields = 0: off */
    int32_t ray_fields;             /* bitmask: 1 u, 2 v, 4 w, 8 theta */
    int32_t moist;                  /* 1 = moist air (FP64 path, flat or terrain): rho q_v, rho q_c,
                                       rho q_r per unit dry mass, transported like scalars (Sec. 3.1)
                                       and diffused with the heat diffusivity of the closure; the
                                       moist EOS p = P00 (R_d rho theta (1 + (R_v/R_d) q_v)/P00)^gamma
                                       (Sec. 2.1, R_v = 461.5); pressure gradient and buoyancy over
                                       1 + q_v + q_c with the buoyancy of the total density
                                       rho (1 + q_v + q_c + q_r) (Eq. mom); App. C's moisture factors
                                       in the substep coefficients; the base state hydrostatic in
                                       the total density with the vapour sounding below; and Kessler
                                       microphysics (Sec. 2.4, Klemp & Wilhelmson 1978 with a Tetens
                                       saturation) after every RK3 step.  0 = dry */
    int32_t n_qknots;               /* moist: piecewise-linear base-state vapour sounding q_v0(z) */
    const double *qknot_z, *qknot_v;   /* host, n_qknots each [m, kg/kg], read during erf_init_grid only */
    double relax_tau, relax_width;  /* open x boundaries as relaxation zones (Sec. 3.8, FP64 path):
                                       within relax_width [m] of an x-edge every prognostic field
                                       (moisture included) relaxes toward the reference state at rate
                                       relax_tau sin^2(pi/2 (1 - d/relax_width)) [1/s], d the distance
                                       to the edge; the reference is the state after
                                       erf_set_initial(_moist) or erf_capture_reference.  0 = off */
    int32_t anelastic;              /* 1 = the anelastic equation set (Sec. 2.2; FP64 path, flat grids,
                                       nx and ny powers of two up to 4096): rho held at the base
                                       density, buoyancy rho0 g (theta - theta0) / theta0, SSP-RK2 steps
                                       (Sec. 3.2) on the slow tendencies with the lagged pressure, each
                                       stage projected by an exact FFT (x, y) + tridiagonal (z) Poisson
                                       solve of dt div(grad psi) = div(rho0 u): rho0 u -= dt grad psi;
                                       p' = p'^n + psi after stage 1 and (p'^n + p'*)/2 + psi after
                                       stage 2 (the field ERF_P_ANELASTIC); erf_set_initial projects
                                       the initial momentum.  No acoustic substeps.  0 = compressible */
} erf_config;

/* Diagnostics (Sec. 4.1.2: mass conserved to machine precision). */
typedef struct {
    double mass;            /* sum rho * cell volume, FP64, fixed reduction order */
    double max_abs_w;       /* max |rho w / rho| over interior w-faces [m/s] */
    double theta_min, theta_max;
    double cfl_acoustic;    /* max (|u| + c) dt / dx over x-faces (horizontal acoustic CFL, Sec. 3.3) */
    int32_t nonfinite;      /* 1 if any state value is NaN/Inf */
    int64_t steps_done;
    int32_t kernels_per_step;   /* kernel nodes in the captured step graph */
} erf_diag;

/* Bytes of device workspace the grid + configuration needs (Sec. 3.4 grid, App. C work arrays). */
erf_status erf_workspace_bytes(const erf_grid_desc *grid, const erf_config *cfg, size_t *bytes);

/* Builds metrics (App. B) and the HSE base state (Sec. 2, Sec. 3.8 Newton-Raphson) inside the
 * caller's workspace on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * Returns ERF_ENOSPACE if workspace_bytes is too small, ERF_EUNSUPPORTED for a subgrid closure
 * over terrain. On success *out owns a host handle. */
erf_status erf_init_grid(const erf_grid_desc *grid, const erf_config *cfg, void *d_workspace,
                         size_t workspace_bytes, void *cuda_stream, erf_handle **out);

/* Initial state from a potential-temperature perturbation at unchanged pressure (Sec. 4.1.2:
 * warm perturbations at constant pressure give negative density perturbations):
 *   theta = theta0 + dtheta, rho theta = rho0 theta0, rho = rho theta / theta,
 *   rho u = u * (face-averaged rho), likewise v and w; walls get Omega = 0.
 * Each pointer may be NULL (zero).  dtheta/u/v are nz*ny*nx, w is (nz+1)*ny*nx, FP64, on the
 * host (is_device = 0) or the device (is_device = 1). */
erf_status erf_set_initial(erf_handle *h, const double *dtheta, const double *u, const double *v,
                           const double *w, int32_t is_device);

/* Moist initial state (config moist = 1): theta = theta0 + dtheta and water vapour q_v (nz*ny*nx,
 * NULL = the base state's q_v0) at unchanged pressure (rho theta (1 + (R_v/R_d) q_v) held at its
 * base-state value), no cloud or rain; velocities as erf_set_initial.  The result is also the
 * reference of the relaxation zones.  ERF_EUNSUPPORTED on a dry handle. */
erf_status erf_set_initial_moist(erf_handle *h, const double *dtheta, const double *qv, const double *u,
                                 const double *v, const double *w, int32_t is_device);

/* The current state becomes the reference of the lateral relaxation zones (after fields were set
 * with erf_set_state).  ERF_EUNSUPPORTED without relaxation zones, ERF_ESTATE before any state. */
erf_status erf_capture_reference(erf_handle *h);

/* Passive-scalar initial state: rho phi = rho phi0 at cells with the current rho (Sec. 3.1,
 * scalar equation).  phi0 is nz*ny*nx FP64 on the host (is_device = 0) or the device.
 * ERF_EUNSUPPORTED unless the handle was configured with tracer = 1. */
erf_status erf_set_tracer_initial(erf_handle *h, const double *phi0, int32_t is_device);

/* Copies one prognostic field (ERF_RHO..ERF_RHOW, ERF_RHOPHI) in, converting from src_dtype
 * (erf_dtype). */
erf_status erf_set_state(erf_handle *h, int32_t field, const void *src, int32_t src_is_device,
                         int32_t src_dtype);

/* Advances nsteps RK3 steps (Sec. 3.1 with App. C substeps), one CUDA-graph launch per step,
 * asynchronously on the bound stream.  ERF_ESTATE before any state was set. */
erf_status erf_rk3_step(erf_handle *h, int32_t nsteps);

/* Copies one field (prognostic or base state) out, converting to dst_dtype. */
erf_status erf_get_state(erf_handle *h, int32_t field, void *dst, int32_t dst_is_device,
                         int32_t dst_dtype);

/* Synchronises the stream and fills *out. Returns ERF_ENONFINITE if the state is not finite. */
erf_status erf_diagnostics(erf_handle *h, erf_diag *out);

/* ---- Learned subgrid closure (an extension of the method; the paper names surrogate models as
 * future work, Sec. 6).  Network 12 -> 64 -> 64 -> 64 -> 9 with SiLU, inputs = resolved velocity
 * gradients (9), dtheta/dx, dtheta/dy, N^2 at cell centres; outputs = kinematic SGS stress
 * (t11, t22, t33, t12, t13, t23) and heat flux (h1, h2, h3), both standardised.
 * Parameter vector (FP32, 9737 values): W1[64][12] b1[64] W2[64][64] b2 W3[64][64] b3 W4[9][64] b4[9].
 * All pointers below are device pointers; every call is asynchronous on cuda_stream. */
typedef struct {
    int32_t epochs, batch;          /* passes over the samples; mini-batch size */
    float lr, beta1, beta2, eps;    /* Adam (Kingma & Ba 2015) */
} erf_train_cfg;

/* Loads a closure blob (host): uint32 magic 0x4D465245 ("ERFM"), uint32 version, then FP32
 * in_mean[12] in_std[12] out_mean[9] out_std[9] params[9737].  The weights are rounded to BF16 on
 * the device for tensor-core inference.  The handle must have been created with
 * closure = ERF_CLOSURE_LEARNED (mixed precision); steps refuse to run (ERF_ESTATE) until this
 * call has succeeded.  Cells whose standardised inputs exceed 6 in magnitude, or whose outputs
 * are not finite, use the Smagorinsky stresses instead. */
erf_status erf_set_closure_weights(erf_handle *h, const void *blob, size_t bytes);

/* The 12 closure inputs of every cell of the current state, d_out [nz*ny*nx][12] (mixed path). */
erf_status erf_closure_features(erf_handle *h, float *d_out);

/* The closure's density-weighted SGS stress and heat flux of the current state at cell centres,
 * d_out9 = 9 planes of nz*ny*nx floats (rho t11, t22, t33, t12, t13, t23, rho h1, h2, h3);
 * *n_fallback (optional, host) receives the number of cells that used Smagorinsky. Syncs. */
erf_status erf_closure_fields(erf_handle *h, float *d_out9, uint32_t *n_fallback);

/* Favre r x r x r box filter of the current (fine, flat, mixed-precision) state into a coarse
 * C-grid state with the same layout conventions (d_rho, d_rhotheta, d_rhou, d_rhov: Nz*Ny*Nx,
 * d_rhow: (Nz+1)*Ny*Nx, FP64, N = n/r) and the SGS targets t_ij, h_j at coarse cells,
 * d_targets [Nz*Ny*Nx][9] (kinematic, same order as the closure outputs). */
erf_status erf_filter_state(erf_handle *h, int32_t r, double *d_rho, double *d_rhotheta, double *d_rhou,
                            double *d_rhov, double *d_rhow, float *d_targets);

/* Bytes of device scratch erf_train_closure / erf_closure_grad need for mini-batch `batch`. */
size_t erf_train_scratch_bytes(int32_t batch);

/* Mini-batch Adam on MSE over n standardised samples (d_X [n][12], d_T [n][9]) in the given
 * order; d_params (9737 FP32) is updated in place; d_losses (optional) receives the loss of each
 * mini-batch.  Deterministic (fixed summation order). */
erf_status erf_train_closure(const erf_train_cfg *cfg, const float *d_X, const float *d_T, int64_t n,
                             float *d_params, float *d_losses, void *d_scratch, size_t scratch_bytes,
                             void *cuda_stream);

/* Loss and gradient of one batch of n samples (no update): d_grad (9737), d_loss (1). */
erf_status erf_closure_grad(const float *d_X, const float *d_T, int32_t n, float *d_params, float *d_grad,
                            float *d_loss, void *d_scratch, size_t scratch_bytes, void *cuda_stream);

/* Per-column mean and standard deviation (0 replaced by 1) of d_A [rows][cols]; and
 * standardisation out = (A - mean)/std. */
erf_status erf_column_stats(const float *d_A, int64_t rows, int32_t cols, float *d_mean, float *d_std,
                            void *cuda_stream);
erf_status erf_standardise(const float *d_A, int64_t rows, int32_t cols, const float *d_mean,
                           const float *d_std, float *d_out, void *cuda_stream);

/* Per-kernel device time of a profiled run. */
typedef struct {
    char name[48];          /* kernel name without the k_ prefix */
    double total_ms;        /* summed CUDA-event time of all its launches */
    int32_t launches;
} erf_kernel_time;

/* Tracing aid (not part of the paper's method): advances nsteps RK3 steps exactly like
 * erf_rk3_step but by direct launches with a CUDA event pair around every kernel on the bound
 * stream, synchronises, and fills up to max_entries per-kernel totals (*n_entries set). */
erf_status erf_profile_steps(erf_handle *h, int32_t nsteps, erf_kernel_time *out, int32_t max_entries,
                             int32_t *n_entries);

/* Allocation-free state reduction.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory (code running inside another framework's memory
 * pool, sandboxes that forbid cudaMalloc, hosts whose HBM is already handed to a fixed arena).
 * It reduces a state the caller already holds in device memory - flat grid, the same layout as
 * erf_get_state, d_dz = the nz cell heights - into d_out[0..4] = {mass, max abs(w) over interior
 * w-faces, theta min, theta max, nonfinite flag (1.0/0.0)} on cuda_stream, with the same fixed
 * reduction order on every call.  The mass weights each cell by dz[k] dx dy, the volume of a
 * flat-grid cell: for a state over terrain (where each column's cell heights differ) the mass it
 * returns is wrong, and erf_diagnostics, which weights by each cell's own height, is the one to
 * use.  It needs no handle and no workspace and calls no allocator:
 * its only scratch is a file-scope device array of ERF_NOALLOC_MAX_PARTS x 5 doubles (2.5 MiB)
 * that every GPU loading the library keeps until the process exits.  Grids of more than
 * ERF_NOALLOC_MAX_PARTS x 4096 cells are rejected with ERF_ENOSPACE.  The first call on a
 * device looks up that array's device address (once per device, with the device current), so
 * make the first call before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (two streams, two host threads) race; serialise them.  Every value a call reads
 * from the array is written by the same call, so nothing needs clearing between calls. */
#define ERF_NOALLOC_MAX_PARTS 65536
erf_status erf_reduce_state_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double dy,
                                    const double *d_dz, const double *d_rho, const double *d_rhotheta,
                                    const double *d_rhou, const double *d_rhov, const double *d_rhow,
                                    double *d_out, void *cuda_stream);

/* ---- x-y pencil decomposition (Sec. 5.1-5.2: the domain is split over ranks, each rank's
 * boundary columns refreshed from its neighbours).  A rank advances its pencil widened by a halo
 * of H columns per sharded side (H at least the columns one RK3 step reaches sideways) and
 * refreshes the halo once per step; these calls move the halo strips.  A column block is the
 * columns [i0, i0+ni) x [j0, j0+nj) (0 <= i0, i0+ni <= nx, likewise j) at every level of every
 * prognostic field - rho, rho theta, rho u, rho v (nz levels each), rho w (nz+1), then rho phi
 * when the handle carries the passive scalar - packed field after field, each [k][jj][ii] with ii
 * fastest, in the path's storage type (FP64 on the FP64 path; the FP32 perturbations from the
 * base state on the mixed path, so a block copied between two handles of the same grid levels
 * and base state is bit-identical).  d_buf is a device buffer owned by the caller, at least
 * erf_column_block_bytes long.  Both copies are asynchronous on the bound stream (capturable);
 * erf_unpack_columns takes effect for the next step.  Errors: ERF_EINVAL for a block outside the
 * grid or NULL pointers, ERF_ESTATE for a pack before any state was set. */
erf_status erf_column_block_bytes(const erf_handle *h, int32_t ni, int32_t nj, size_t *bytes);
erf_status erf_pack_columns(erf_handle *h, int32_t i0, int32_t ni, int32_t j0, int32_t nj, void *d_buf);
erf_status erf_unpack_columns(erf_handle *h, int32_t i0, int32_t ni, int32_t j0, int32_t nj, const void *d_buf);

/* Runtime options (no counterpart in the paper).
 *   ERF_OPT_TMA_STENCILS: 1 (default) stages the 3D stencils of the mixed-precision flux kernels
 *   in shared memory with TMA tile loads where the grid allows it (nx % 4 == 0, nx >= 64,
 *   ny >= 16, nz >= 16); 0 uses plain loads.  Both give bit-identical results.  A TMA wait that
 *   gives up makes the next erf_diagnostics return ERF_ECUDA.
 *   ERF_OPT_COLUMN_FUSION: how the mixed-precision substep runs the explicit vertical part
 *   (App. C rows 3-4): 1 inside the column sweep of the vertical solve, one thread per column;
 *   0 as a per-cell kernel before the sweep; -1 (default) fused when nx * ny >= 2^17.  Both give
 *   bit-identical results.
 *   ERF_OPT_WARP_COLUMNS: how the FP64 path builds the stage's vertical acoustic system (App. C):
 *   1 one warp per column (the lanes form the levels' coefficients at once, one lane runs the LU
 *   recurrence; for grids with few columns such as 2D slabs, nz <= 256), 0 one thread per column,
 *   -1 (default) one warp per column below 2^15 columns.  Both give bit-identical results.
 * erf_set_option drops the captured step graph; erf_get_option reports whether the option is in
 * effect (1 if the TMA kernels run, 1 if the fused column sweep runs, 1 if warps build the columns). */
typedef enum { ERF_OPT_TMA_STENCILS = 1, ERF_OPT_COLUMN_FUSION = 2, ERF_OPT_WARP_COLUMNS = 3 } erf_option;
erf_status erf_set_option(erf_handle *h, int32_t option, int64_t value);
erf_status erf_get_option(erf_handle *h, int32_t option, int64_t *value);

/* Self-test of the bounded device-side waits (no counterpart in the paper): launches one block
 * that arms an mbarrier with a byte count no copy delivers and polls it at most max_polls times.
 * *timed_out = 1 when the wait gave up and reported it (the expected outcome).  d_flag is one
 * device word owned by the caller; the context stays usable.  Synchronises cuda_stream. */
erf_status erf_selftest_wait_timeout(int32_t max_polls, unsigned *d_flag, void *cuda_stream, int32_t *timed_out);

/* Self-test of the tensor-core (tcgen05) path used by the learned closure: one CTA runs MMAs of
 * the network's operand shapes (M = 128; K = 64 with N = 64 and N = 16; K = 16 with N = 64) on
 * exact small-integer BF16 data through the same shared-memory layouts and descriptors, reads
 * the TMEM accumulators back and compares every output with integer loops.  d_words is two
 * int32 device words owned by the caller (scratch).  *mismatches = outputs that differ (0 when
 * the path is correct); *timed_out = 1 if the bounded wait on the MMAs gave up.  Synchronises
 * cuda_stream. */
erf_status erf_selftest_tensor_cores(int32_t *d_words, void *cuda_stream, int32_t *mismatches, int32_t *timed_out);

/* Message of the last failed call on h (or of the last failed erf_init_grid if h is NULL). */
const char *erf_last_error(const erf_handle *h);

/* Frees the host handle and the library's private stream/graph; the workspace stays the caller's. */
void erf_destroy(erf_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* ERF_GB300_H */
