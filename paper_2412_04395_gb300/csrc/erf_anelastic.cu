// The anelastic equation set (Sec. 2.2) and its time integration (Sec. 3.2) on the FP64 path:
// SSP-RK2 (Shu & Osher 1988) on the slow tendencies of the compressible kernels (rho held at the
// base density, the pressure perturbation the projection's, buoyancy rho0 g (theta - theta0) /
// theta0), each stage followed by a projection that solves dt div(grad psi) = div(rho0 u**) and
// sets rho0 u = rho0 u** - dt grad psi.  The Poisson problem of the C-grid is solved exactly: an
// FFT in x and y (periodic) turns it into one tridiagonal system in z per horizontal wavenumber
// (walls: no flux).  The FFT is a radix-2 transform in shared memory, one CTA per line: x-lines
// are contiguous, y-lines strided by nx.  Flat grids, nx and ny powers of two.
#include <cuda_runtime.h>

#include "erf_launch.h"

namespace erfk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ unsigned bitrev(unsigned q, int logn) { return logn == 0 ? 0u : __brev(q) >> (32 - logn); }

// the stage's EOS-free start: p' = the projection's pressure, theta = rho theta / rho
__global__ void k_anel_begin(Geo g, const double *rt, const double *rho, const double *pa, double *pp, double *th) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    pp[c] = pa[c];
    th[c] = rt[c] * rcp_d(rho[c]);
}

// S = S^n + a R1 + b R for rho theta and the momenta (rho stays rho0; the wall rows of rho w keep
// their zero tendency)
__global__ void k_anel_stage(Geo g, F5 st, CF5 sn, CF5 R1, CF5 R, double a, double b) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    if (n < g.nc) {
        st.t[n] = sn.t[n] + (a * R1.t[n] + b * R.t[n]);
        st.u[n] = sn.u[n] + (a * R1.u[n] + b * R.u[n]);
        st.v[n] = sn.v[n] + (a * R1.v[n] + b * R.v[n]);
    }
    st.w[n] = sn.w[n] + (a * R1.w[n] + b * R.w[n]);
}

// right-hand side div(rho0 u**) / dt of the Poisson problem, as a complex field (imaginary part 0)
__global__ void k_anel_div(Geo g, const double *mu, const double *mv, const double *mw, double rdt, double2 *cw) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    double d = (__ldg(mu + cixw(g, i + 1, j, k)) - __ldg(mu + c)) * g.rdx
             + (__ldg(mv + cixw(g, i, j + 1, k)) - __ldg(mv + c)) * g.rdy
             + (__ldg(mw + c + g.nxy) - __ldg(mw + c)) * g.rdzeta[k];
    cw[c] = make_double2(d * rdt, 0.0);
}

// one radix-2 FFT of length n = 2^logn per CTA (decimation in time, bit-reversed load):
// axis 0 transforms the x-lines (nz * ny of them), axis 1 the y-lines (nz * nx, stride nx);
// dir -1 forward, +1 inverse (scaled by 1/n); tw[m] = exp(-2 pi i m / n), m < n/2
__global__ void k_fft(double2 *data, const double2 *tw, int n, int logn, int dir, int axis, int nx, int ny) {
    extern __shared__ double2 buf[];
    const long long t = blockIdx.x;
    long long base, es;
    if (axis == 0) {
        base = t * nx;
        es = 1;
    } else {
        const long long k = t / nx, i = t % nx;
        base = k * (long long)nx * ny + i;
        es = nx;
    }
    for (int q = threadIdx.x; q < n; q += blockDim.x) buf[bitrev((unsigned)q, logn)] = data[base + q * es];
    __syncthreads();
    for (int s = 1; s <= logn; ++s) {
        const int half = 1 << (s - 1);
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int jj = b & (half - 1), grp = b >> (s - 1);
            const int i0 = grp * 2 * half + jj, i1 = i0 + half;
            double2 w = tw[jj * (n >> s)];
            if (dir > 0) w.y = -w.y;
            const double2 v = cmul(w, buf[i1]), u = buf[i0];
            buf[i0] = make_double2(u.x + v.x, u.y + v.y);
            buf[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    const double sc = dir > 0 ? 1.0 / n : 1.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const double2 v = buf[q];
        data[base + q * es] = make_double2(v.x * sc, v.y * sc);
    }
}

// per horizontal wavenumber (i, j): the tridiagonal system in z of the transformed Poisson
// problem, lo_k psi_{k-1} + (a - lo_k - up_k) psi_k + up_k psi_{k+1} = r_k with
// a = lamx_i + lamy_j, lo_k = 1/(dz_k dzc_k), up_k = 1/(dz_k dzc_{k+1}) (zero at the walls);
// the (0, 0) mode takes psi_0 = 0.  cp: nc scratch values.
__global__ void k_poisson_tri(Geo g, const double *lamx, const double *lamy, double2 *cw, double *cp) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nxy) return;
    const int i = (int)(n % g.nx), j = (int)(n / g.nx);
    const double a = lamx[i] + lamy[j];
    const int nz = g.nz;
    auto lo = [&](int k) { return k >= 1 ? g.rdzeta[k] * g.rdzc[k] : 0.0; };
    auto up = [&](int k) { return k <= nz - 2 ? g.rdzeta[k] * g.rdzc[k + 1] : 0.0; };
    const bool zero_mode = (i == 0 && j == 0);
    double d0 = a - lo(0) - up(0), u0 = up(0);
    double2 r0 = cw[n];
    if (zero_mode) { d0 = 1.0; u0 = 0.0; r0 = make_double2(0.0, 0.0); }
    double cprev = u0 / d0;
    double2 dprev = make_double2(r0.x / d0, r0.y / d0);
    cp[n] = cprev;
    cw[n] = dprev;
    for (int k = 1; k < nz; ++k) {
        const long long c = n + (long long)k * g.nxy;
        const double l = lo(k), m = a - l - up(k) - l * cprev;
        const double2 r = cw[c];
        cprev = up(k) / m;
        dprev = make_double2((r.x - l * dprev.x) / m, (r.y - l * dprev.y) / m);
        cp[c] = cprev;
        cw[c] = dprev;
    }
    double2 x = dprev;
    for (int k = nz - 2; k >= 0; --k) {
        const long long c = n + (long long)k * g.nxy;
        const double2 d = cw[c];
        x = make_double2(d.x - cp[c] * x.x, d.y - cp[c] * x.y);
        cw[c] = x;
    }
}

// rho0 u -= dt grad psi at x-, y- and interior w-faces (psi = the real part of cw); and the new
// pressure: stage 1  p' = p'^n + psi  (written to pa and pa1), stage 2  p' = (p'^n + p'*)/2 + psi
__global__ void k_anel_correct(Geo g, const double2 *cw, double dt, double *mu, double *mv, double *mw,
                               const double *pan, double *pa1, double *pa, int stage) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nw) return;
    int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / g.nxy);
    if (k < g.nz) {
        const double p0 = cw[n].x;
        mu[n] -= dt * ((p0 - cw[cixw(g, i - 1, j, k)].x) * g.rdx);
        mv[n] -= dt * ((p0 - cw[cixw(g, i, j - 1, k)].x) * g.rdy);
        if (stage == 1) {
            const double p = pan[n] + p0;
            pa1[n] = p;
            pa[n] = p;
        } else if (stage == 2) {
            pa[n] = 0.5 * (pan[n] + pa1[n]) + p0;
        }
    }
    if (k >= 1 && k < g.nz) mw[n] -= dt * ((cw[n].x - cw[n - g.nxy].x) * g.rdzc[k]);
}

// initial state: rho = rho0, rho theta = rho0 (theta0 + dtheta)
__global__ void k_anel_init(Geo g, const double *dth, double *rho, double *rt) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    long long b = bix(g, i, j, k);
    rho[c] = g.rho0[b];
    rt[c] = g.rho0[b] * (g.th0[b] + (dth ? dth[c] : 0.0));
}

static inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_anel_begin(const Geo &g, const double *rt, const double *rho, const double *pa, double *pp, double *th,
                       cudaStream_t s) {
    ProfLaunch pl("anel_begin", s);
    k_anel_begin<<<nb(g.nc, 256), 256, 0, s>>>(g, rt, rho, pa, pp, th);
}
void launch_anel_stage(const Geo &g, F5 st, CF5 sn, CF5 R1, CF5 R, double a, double b, cudaStream_t s) {
    ProfLaunch pl("anel_stage", s);
    k_anel_stage<<<nb(g.nw, 256), 256, 0, s>>>(g, st, sn, R1, R, a, b);
}
void launch_anel_init(const Geo &g, const double *dth, double *rho, double *rt, cudaStream_t s) {
    ProfLaunch pl("anel_init", s);
    k_anel_init<<<nb(g.nc, 256), 256, 0, s>>>(g, dth, rho, rt);
}

static int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
void launch_anel_project(const Geo &g, const AnelWork &w, double dt, double *mu, double *mv, double *mw, int stage,
                         cudaStream_t s) {
    {
        ProfLaunch pl("anel_div", s);
        k_anel_div<<<nb(g.nc, 256), 256, 0, s>>>(g, mu, mv, mw, 1.0 / dt, w.cw);
    }
    const int lx = ilog2(g.nx), ly = ilog2(g.ny);
    const int tx = g.nx >= 512 ? 256 : (g.nx / 2 > 32 ? g.nx / 2 : 32);
    const int ty = g.ny >= 512 ? 256 : (g.ny / 2 > 32 ? g.ny / 2 : 32);
    {
        ProfLaunch pl("anel_fft", s);
        k_fft<<<(unsigned)(g.nz * (long long)g.ny), tx, g.nx * sizeof(double2), s>>>(w.cw, w.twx, g.nx, lx, -1, 0, g.nx, g.ny);
        if (g.ny > 1)
            k_fft<<<(unsigned)(g.nz * (long long)g.nx), ty, g.ny * sizeof(double2), s>>>(w.cw, w.twy, g.ny, ly, -1, 1, g.nx, g.ny);
    }
    {
        ProfLaunch pl("anel_tri", s);
        k_poisson_tri<<<nb(g.nxy, 128), 128, 0, s>>>(g, w.lamx, w.lamy, w.cw, w.cp);
    }
    {
        ProfLaunch pl("anel_fft", s);
        if (g.ny > 1)
            k_fft<<<(unsigned)(g.nz * (long long)g.nx), ty, g.ny * sizeof(double2), s>>>(w.cw, w.twy, g.ny, ly, 1, 1, g.nx, g.ny);
        k_fft<<<(unsigned)(g.nz * (long long)g.ny), tx, g.nx * sizeof(double2), s>>>(w.cw, w.twx, g.nx, lx, 1, 0, g.nx, g.ny);
    }
    {
        ProfLaunch pl("anel_correct", s);
        k_anel_correct<<<nb(g.nw, 256), 256, 0, s>>>(g, w.cw, dt, mu, mv, mw, w.pan, w.pa1, w.pa, stage);
    }
}

// lets the FFT use up to 64 KB of shared memory (lines of up to 4096 points)
bool anel_fft_setup() {
    return cudaFuncSetAttribute(k_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * (int)sizeof(double2)) ==
           cudaSuccess;
}

}  // namespace erfk
