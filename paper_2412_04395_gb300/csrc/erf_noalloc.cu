// Allocation-free variant of the state reduction behind erf_diagnostics.
//
// Some callers cannot allocate device memory at all: code that runs inside another framework's
// memory pool or a sandbox that forbids cudaMalloc, hosts that have handed every byte of HBM to
// a pre-sized arena, or call sites that must not allocate while a long-running job is resident.
// They can still hand over the arrays they already own.  erf_reduce_state_noalloc reduces such a
// state with no workspace: its only scratch (the per-block partial results of the first
// reduction pass) lives in the file-scope device array below, sized for at most
// ERF_NOALLOC_MAX_PARTS blocks.  Every GPU that loads the library holds this array until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/erf.h"

namespace {

constexpr int NA_BS = 256;                          // threads per block
constexpr long long NA_ITEMS = 16;                  // cells per thread
constexpr long long NA_CELLS_PER_BLOCK = NA_BS * NA_ITEMS;
constexpr int NA_FIELDS = 5;                        // mass, max|w|, theta min, theta max, nonfinite

// scratch: partial results of the first pass, NA_FIELDS doubles per block
static __device__ __align__(256) double g_noalloc_parts[ERF_NOALLOC_MAX_PARTS * NA_FIELDS];

struct Dev {
    std::once_flag once;
    double *parts = nullptr;
    cudaError_t err = cudaSuccess;
};
constexpr int NA_MAX_DEVICES = 64;
Dev g_dev[NA_MAX_DEVICES];

// pass 1: each block reduces NA_CELLS_PER_BLOCK consecutive cells in a fixed order
__global__ void k_na_partial(int nx, int ny, int nz, double dxdy, const double *dz, const double *rho,
                             const double *rt, const double *ru, const double *rv, const double *rw,
                             double *parts) {
    __shared__ double s[NA_FIELDS][NA_BS];
    const long long nxy = (long long)nx * ny, nc = nxy * nz;
    const int t = threadIdx.x;
    double mass = 0.0, wmax = 0.0, tmn = 1e300, tmx = -1e300, nf = 0.0;
    long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
    for (long long q = 0; q < NA_ITEMS; ++q) {
        long long c = base + q * NA_BS + t;
        if (c >= nc) break;
        int k = (int)(c / nxy);
        double r = rho[c], th = rt[c] / r;
        mass += r * dz[k] * dxdy;
        tmn = fmin(tmn, th);
        tmx = fmax(tmx, th);
        if (!isfinite(r) || !isfinite(rt[c]) || !isfinite(ru[c]) || !isfinite(rv[c]) || !isfinite(rw[c])) nf = 1.0;
        if (k > 0) {   // interior w-face k (bottom face of cell k)
            double rb = 0.5 * (rho[c - nxy] + r);
            wmax = fmax(wmax, fabs(rw[c] / rb));
        }
        if (k == nz - 1 && !isfinite(rw[c + nxy])) nf = 1.0;
    }
    s[0][t] = mass; s[1][t] = wmax; s[2][t] = tmn; s[3][t] = tmx; s[4][t] = nf;
    __syncthreads();
    for (int h = NA_BS / 2; h > 0; h >>= 1) {
        if (t < h) {
            s[0][t] += s[0][t + h];
            s[1][t] = fmax(s[1][t], s[1][t + h]);
            s[2][t] = fmin(s[2][t], s[2][t + h]);
            s[3][t] = fmax(s[3][t], s[3][t + h]);
            s[4][t] = fmax(s[4][t], s[4][t + h]);
        }
        __syncthreads();
    }
    if (t == 0)
        for (int f = 0; f < NA_FIELDS; ++f) parts[(long long)blockIdx.x * NA_FIELDS + f] = s[f][0];
}

// pass 2: one thread combines the partials in block order
__global__ void k_na_final(const double *parts, int nb, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mass = 0.0, wmax = 0.0, tmn = 1e300, tmx = -1e300, nf = 0.0;
    for (int b = 0; b < nb; ++b) {
        const double *p = parts + (long long)b * NA_FIELDS;
        mass += p[0];
        wmax = fmax(wmax, p[1]);
        tmn = fmin(tmn, p[2]);
        tmx = fmax(tmx, p[3]);
        nf = fmax(nf, p[4]);
    }
    out[0] = mass; out[1] = wmax; out[2] = tmn; out[3] = tmx; out[4] = nf;
}

}  // namespace

extern "C" erf_status erf_reduce_state_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double dy,
                                               const double *d_dz, const double *d_rho, const double *d_rhotheta,
                                               const double *d_rhou, const double *d_rhov, const double *d_rhow,
                                               double *d_out, void *cuda_stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0) || !(dy > 0.0)) return ERF_EINVAL;
    if (!d_dz || !d_rho || !d_rhotheta || !d_rhou || !d_rhov || !d_rhow || !d_out) return ERF_EINVAL;
    long long nc = (long long)nx * ny * nz;
    long long nb = (nc + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK;
    if (nb > ERF_NOALLOC_MAX_PARTS) return ERF_ENOSPACE;   // grid larger than the static scratch covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return ERF_ECUDA;
    // set-up, once per device with that device current: the device address of the static
    // scratch (its host-side name is only a stand-in and must never reach a kernel)
    Dev &D = g_dev[dev];
    std::call_once(D.once, [&D]() {
        D.err = cudaGetSymbolAddress(reinterpret_cast<void **>(&D.parts), g_noalloc_parts);
    });
    if (D.err != cudaSuccess || !D.parts) return ERF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    k_na_partial<<<(unsigned)nb, NA_BS, 0, s>>>(nx, ny, nz, dx * dy, d_dz, d_rho, d_rhotheta, d_rhou, d_rhov,
                                                d_rhow, D.parts);
    k_na_final<<<1, 32, 0, s>>>(D.parts, (int)nb, d_out);
    return cudaGetLastError() == cudaSuccess ? ERF_OK : ERF_ECUDA;
}
