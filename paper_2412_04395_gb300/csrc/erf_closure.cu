// Learned subgrid closure: features, BF16 tensor-core inference with Smagorinsky fallback, the
// 4x box filter that makes training targets, and the weight upload.
//
// Inference maps each cell's 12 features (resolved velocity gradients, dtheta/dx, dtheta/dy, N^2)
// through 12 -> 64 -> 64 -> 64 -> 9 (SiLU) to the kinematic SGS stress and heat flux.  A warp
// takes 32 cells (one per lane for the features and the store), as two 16-row tiles: the
// 16 x 16 feature tiles (12 + 4 zero columns) and every hidden activation tile live in BF16
// mma.sync fragments (m16n8k16, FP32 accumulate); the accumulator fragments of two adjacent
// n-tiles are exactly the A fragment of the next k-tile, so activations never leave registers
// between layers, and each B fragment loaded from shared memory feeds both tiles.  Weights sit
// in shared memory in [out][in] row-major BF16 (the "col" B-fragment order of the instruction),
// rows padded to 24 / 72 elements so that the eight rows one B load touches fall in distinct
// banks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/erf.h"
#include "erf_closure.h"
#include "erf_dev.cuh"
#include "erf_launch.h"
#include "erf_mixed.h"

namespace erfk {

// device weight block (built from a blob by k_cl_prepare)
struct ClDev {
    const __nv_bfloat16 *W1;   // [64][16]  (inputs padded with zeros)
    const __nv_bfloat16 *W2;   // [64][64]
    const __nv_bfloat16 *W3;   // [64][64]
    const __nv_bfloat16 *W4;   // [16][64]  (outputs padded with zero rows)
    const float *b;            // b1[64] b2[64] b3[64] b4[16]
    const float *stats;        // in_mean[12] in_std[12] out_mean[9] out_std[9]
};
constexpr int CL_B_F32 = 64 * 3 + 16;

__global__ void k_cl_prepare(const float *blob, __nv_bfloat16 *w, float *b, float *stats) {
    const float *st = blob;                 // 42 stats
    const float *p = blob + 2 * CL_NIN + 2 * CL_NOUT;
    const float *W1 = p, *b1 = W1 + 64 * 12, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64, *b3 = W3 + 64 * 64;
    const float *W4 = b3 + 64, *b4 = W4 + 9 * 64;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * CL_NIN + 2 * CL_NOUT) stats[t] = st[t];
    if (t < 64 * 16) { int o = t / 16, i = t % 16; w[t] = __float2bfloat16_rn(i < 12 ? W1[o * 12 + i] : 0.f); }
    if (t < 64 * 64) {
        w[1024 + t] = __float2bfloat16_rn(W2[t]);
        w[1024 + 4096 + t] = __float2bfloat16_rn(W3[t]);
    }
    if (t < 16 * 64) { int o = t / 64, i = t % 64; w[1024 + 8192 + t] = __float2bfloat16_rn(o < 9 ? W4[o * 64 + i] : 0.f); }
    if (t < 64) { b[t] = b1[t]; b[64 + t] = b2[t]; b[128 + t] = b3[t]; }
    if (t < 16) b[192 + t] = t < 9 ? b4[t] : 0.f;
}

__device__ __forceinline__ float fv(const Geo &g, const float *f, int i, int j, int k) {
    return __ldg(f + cixw(g, i, j, kref(k, g.nz)));
}

// the 12 inputs at cell (i,j,k); also returns dtheta/dz (for the fallback heat flux).  Neighbour
// loads use offsets from the cell index: periodic wrap in x and y, the reflected (clamped)
// neighbour level in z.
struct VelIn {
    const float *ux, *vy, *wz, *thp;
};
__device__ void cl_features(const Geo &g, const MxBase &mb, const VelIn &v, int i, int j, int k, float *f,
                            float &dthdz) {
    const float rdx = mb.rdx, rdy = mb.rdy;
    const long long nx = g.nx, nxy = g.nxy;
    const long long c = ((long long)k * g.ny + j) * nx + i;
    const long long oxp = i + 1 < g.nx ? 1 : 1 - nx, oxm = i > 0 ? -1 : nx - 1;
    const long long oyp = j + 1 < g.ny ? nx : nx - nxy, oym = j > 0 ? -nx : nxy - nx;
    const long long okp = k + 1 < g.nz ? nxy : 0, okm = k > 0 ? -nxy : 0;
    auto L = [](const float *p, long long o) { return __ldg(p + o); };
    auto uc = [&](long long o) { return 0.5f * (L(v.ux, c + o) + L(v.ux, c + o + oxp)); };
    auto vc = [&](long long o) { return 0.5f * (L(v.vy, c + o) + L(v.vy, c + o + oyp)); };
    auto wc = [&](long long o) { return 0.5f * (L(v.wz, c + o) + L(v.wz, c + o + nxy)); };
    const float rz = mb.r2dzf[k];
    f[0] = (L(v.ux, c + oxp) - L(v.ux, c)) * rdx;
    f[1] = (uc(oyp) - uc(oym)) * 0.5f * rdy;
    f[2] = (uc(okp) - uc(okm)) * rz;
    f[3] = (vc(oxp) - vc(oxm)) * 0.5f * rdx;
    f[4] = (L(v.vy, c + oyp) - L(v.vy, c)) * rdy;
    f[5] = (vc(okp) - vc(okm)) * rz;
    f[6] = (wc(oxp) - wc(oxm)) * 0.5f * rdx;
    f[7] = (wc(oyp) - wc(oym)) * 0.5f * rdy;
    f[8] = (L(v.wz, c + nxy) - L(v.wz, c)) * mb.rdzf[k];
    f[9] = (L(v.thp, c + oxp) - L(v.thp, c + oxm)) * 0.5f * rdx;
    f[10] = (L(v.thp, c + oyp) - L(v.thp, c + oym)) * 0.5f * rdy;
    int kl = k > 0 ? k - 1 : 0, ku = k < g.nz - 1 ? k + 1 : g.nz - 1;
    dthdz = (mx_dth0(mb, ku, kl) + L(v.thp, c + okp) - L(v.thp, c + okm)) * rz;
    f[11] = mb.gth0f[k] * dthdz;
}

__device__ __forceinline__ unsigned pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // .x = a (low half), .y = b
    return *reinterpret_cast<unsigned *>(&h);
}
__device__ __forceinline__ void mma16816(float *d, const unsigned *a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// SiLU x sigma(x) = h (1 + tanh h), h = x/2: one MUFU operation (tanh.approx.f32, relative error
// about 2^-11) instead of an exponential and a reciprocal.  The activation is rounded to BF16
// (2^-9) right after, and the inference error against a BF16-emulating FP64 network stays at
// 2e-5 .. 2e-4 relative L2 (measured; the test bound is 5e-3).
__device__ __forceinline__ float silu_dev(float x) {
    float h = 0.5f * x, t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// Learned SGS stress/heat flux at every cell (mixed path), with Smagorinsky as the per-cell
// fallback and backscatter limited to half the Smagorinsky transfer.  Persistent blocks of 4 warps load
// the weights into shared memory once and then take 32-cell tiles in turn; each warp runs its
// tile as two m16 tiles through every layer, reusing each B fragment for both.  The bias is the
// accumulator's initial value.
// out: 9 planes of nc floats: rho t11, rho t22, rho t33, rho t12, rho t13, rho t23, rho h1..h3.
constexpr int CLW = 4;
constexpr int LD1 = 24, LDH = 72;   // padded shared-memory row lengths (bank-conflict-free B loads)
constexpr int SW_W1 = 0, SW_W2 = 64 * LD1, SW_W3 = SW_W2 + 64 * LDH, SW_W4 = SW_W3 + 64 * LDH;
constexpr int SW_TOTAL = SW_W4 + 16 * LDH;
__global__ void __launch_bounds__(CLW * 32, 4) k_cl_infer(Geo g, MxBase mb, Phys ph, ClDev cl, VelIn v,
                                                       const float *dr, float *out, unsigned *nfallback) {
    __shared__ __align__(16) __nv_bfloat16 sW[SW_TOTAL];
    __shared__ float sb[CL_B_F32];
    __shared__ float sst[2 * CL_NIN + 2 * CL_NOUT];   // in_mean, 1/in_std, out_mean, out_std
    __shared__ __align__(16) float sF[CLW][32][17];   // standardised features, then outputs
    __shared__ float sMisc[CLW][32][19];              // fallback stresses/fluxes, rho, flag, S_ij, bound
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int q = tid; q < 64 * 16; q += blockDim.x) sW[SW_W1 + (q / 16) * LD1 + q % 16] = cl.W1[q];
    for (int q = tid; q < 64 * 64; q += blockDim.x) {
        sW[SW_W2 + (q / 64) * LDH + q % 64] = cl.W2[q];
        sW[SW_W3 + (q / 64) * LDH + q % 64] = cl.W3[q];
    }
    for (int q = tid; q < 16 * 64; q += blockDim.x) sW[SW_W4 + (q / 64) * LDH + q % 64] = cl.W4[q];
    for (int q = tid; q < CL_B_F32; q += blockDim.x) sb[q] = cl.b[q];
    for (int q = tid; q < 2 * CL_NIN + 2 * CL_NOUT; q += blockDim.x)
        sst[q] = (q >= CL_NIN && q < 2 * CL_NIN) ? 1.f / cl.stats[q] : cl.stats[q];
    __syncthreads();
    const float *in_mu = sst, *in_rsd = sst + 12, *out_mu = sst + 24, *out_sd = sst + 33;
    const float rPr = mb.rPr;
    const int gr = lane >> 2, tc = lane & 3;   // fragment coordinates: row, column pair
    const long long ntiles = (g.nc + 31) / 32;
    for (long long tile = (long long)blockIdx.x * CLW + warp; tile < ntiles; tile += (long long)gridDim.x * CLW) {
        const long long c0 = tile * 32;
        // 1. features of 32 cells (one per lane), standardised; fallback flag on |z| > 6
        {
            long long c = c0 + lane;
            float *m = sMisc[warp][lane];
            int fb = 0;
            if (c < g.nc) {
                unsigned row = (unsigned)(c / g.nx);
                int i = (int)(c - (long long)row * g.nx);
                int j = (int)(row % (unsigned)g.ny), k = (int)(row / (unsigned)g.ny);
                float f[12], dthdz;
                cl_features(g, mb, v, i, j, k, f, dthdz);
                for (int q = 0; q < 12; ++q) {
                    float z = (f[q] - in_mu[q]) * in_rsd[q];
                    if (!(fabsf(z) <= 6.f)) fb = 1;
                    sF[warp][lane][q] = z;
                }
                // Smagorinsky fallback at the cell centre
                float s11 = f[0], s22 = f[4], s33 = f[8];
                float s12 = 0.5f * (f[1] + f[3]), s13 = 0.5f * (f[2] + f[6]), s23 = 0.5f * (f[5] + f[7]);
                float rho = mb.rho0f[k] + dr[c];
                float SS = s11 * s11 + s22 * s22 + s33 * s33 + 2.f * (s12 * s12 + s13 * s13 + s23 * s23);
                float mu = rho * mb.delta2f[k] * sqrtf(2.f * SS);
                float tr = (s11 + s22 + s33) * (1.f / 3.f);
                m[0] = -2.f * mu * (s11 - tr); m[1] = -2.f * mu * (s22 - tr); m[2] = -2.f * mu * (s33 - tr);
                m[3] = -2.f * mu * s12; m[4] = -2.f * mu * s13; m[5] = -2.f * mu * s23;
                m[6] = -mu * rPr * f[9]; m[7] = -mu * rPr * f[10]; m[8] = -mu * rPr * dthdz;
                m[9] = rho;
                m[11] = s11; m[12] = s22; m[13] = s33; m[14] = s12; m[15] = s13; m[16] = s23;
                // backscatter bound: the learned transfer -t_ij S_ij may not fall below -1/2 of
                // the Smagorinsky transfer (both density-weighted)
                float ps = -(m[0] * s11 + m[1] * s22 + m[2] * s33 + 2.f * (m[3] * s12 + m[4] * s13 + m[5] * s23));
                m[17] = -0.5f * ps;
            } else {
                for (int q = 0; q < 12; ++q) sF[warp][lane][q] = 0.f;
                m[9] = 0.f;
            }
            for (int q = 12; q < 16; ++q) sF[warp][lane][q] = 0.f;
            m[10] = (float)fb;
        }
        __syncwarp();
        // 2. MLP on tensor cores
        unsigned a[2][4][4];   // [m-tile][k-tile][reg]
        for (int mt = 0; mt < 2; ++mt) {
            const float *r0 = sF[warp][mt * 16 + gr], *r1 = sF[warp][mt * 16 + gr + 8];
            a[mt][0][0] = pack_bf16(r0[2 * tc], r0[2 * tc + 1]);
            a[mt][0][1] = pack_bf16(r1[2 * tc], r1[2 * tc + 1]);
            a[mt][0][2] = pack_bf16(r0[2 * tc + 8], r0[2 * tc + 9]);
            a[mt][0][3] = pack_bf16(r1[2 * tc + 8], r1[2 * tc + 9]);
        }
        auto hidden = [&](int woff, int ldw, int nkt, const float *bias) {
            float acc[2][8][4];
            for (int nt = 0; nt < 8; ++nt) {
                float bl = bias[nt * 8 + 2 * tc], bh = bias[nt * 8 + 2 * tc + 1];
                for (int mt = 0; mt < 2; ++mt) {
                    acc[mt][nt][0] = bl; acc[mt][nt][1] = bh; acc[mt][nt][2] = bl; acc[mt][nt][3] = bh;
                }
                const __nv_bfloat16 *wr = sW + woff + (nt * 8 + gr) * ldw;
                for (int kt = 0; kt < nkt; ++kt) {
                    unsigned b0 = *reinterpret_cast<const unsigned *>(wr + kt * 16 + 2 * tc);
                    unsigned b1 = *reinterpret_cast<const unsigned *>(wr + kt * 16 + 2 * tc + 8);
                    mma16816(acc[0][nt], a[0][kt], b0, b1);
                    mma16816(acc[1][nt], a[1][kt], b0, b1);
                }
            }
            for (int mt = 0; mt < 2; ++mt)
                for (int kt = 0; kt < 4; ++kt) {
                    const float *lo = acc[mt][2 * kt], *hi = acc[mt][2 * kt + 1];
                    a[mt][kt][0] = pack_bf16(silu_dev(lo[0]), silu_dev(lo[1]));
                    a[mt][kt][1] = pack_bf16(silu_dev(lo[2]), silu_dev(lo[3]));
                    a[mt][kt][2] = pack_bf16(silu_dev(hi[0]), silu_dev(hi[1]));
                    a[mt][kt][3] = pack_bf16(silu_dev(hi[2]), silu_dev(hi[3]));
                }
        };
        hidden(SW_W1, LD1, 1, sb);
        hidden(SW_W2, LDH, 4, sb + 64);
        hidden(SW_W3, LDH, 4, sb + 128);
        // output layer: 2 n-tiles of 8 (9 valid columns)
        float y[2][2][4];
        for (int nt = 0; nt < 2; ++nt) {
            float bl = sb[192 + nt * 8 + 2 * tc], bh = sb[192 + nt * 8 + 2 * tc + 1];
            for (int mt = 0; mt < 2; ++mt) {
                y[mt][nt][0] = bl; y[mt][nt][1] = bh; y[mt][nt][2] = bl; y[mt][nt][3] = bh;
            }
            const __nv_bfloat16 *wr = sW + SW_W4 + (nt * 8 + gr) * LDH;
            for (int kt = 0; kt < 4; ++kt) {
                unsigned b0 = *reinterpret_cast<const unsigned *>(wr + kt * 16 + 2 * tc);
                unsigned b1 = *reinterpret_cast<const unsigned *>(wr + kt * 16 + 2 * tc + 8);
                mma16816(y[0][nt], a[0][kt], b0, b1);
                mma16816(y[1][nt], a[1][kt], b0, b1);
            }
        }
        __syncwarp();
        for (int mt = 0; mt < 2; ++mt)
            for (int nt = 0; nt < 2; ++nt) {
                int col = nt * 8 + 2 * tc;
                float *r0 = sF[warp][mt * 16 + gr], *r1 = sF[warp][mt * 16 + gr + 8];
                r0[col] = y[mt][nt][0];
                r0[col + 1] = y[mt][nt][1];
                r1[col] = y[mt][nt][2];
                r1[col + 1] = y[mt][nt][3];
            }
        __syncwarp();
        // 3. de-standardise, fallback, density weighting, store (one cell per lane, coalesced)
        {
            long long c = c0 + lane;
            if (c < g.nc) {
                const float *m = sMisc[warp][lane];
                int use_fb = m[10] != 0.f;
                float o[9];
                for (int q = 0; q < 9; ++q) {
                    o[q] = sF[warp][lane][q] * out_sd[q] + out_mu[q];
                    if (!isfinite(o[q])) use_fb = 1;
                }
                float rho = m[9];
                for (int q = 0; q < 9; ++q) o[q] *= rho;
                float pl = -(o[0] * m[11] + o[1] * m[12] + o[2] * m[13] + 2.f * (o[3] * m[14] + o[4] * m[15] + o[5] * m[16]));
                if (pl < m[17]) {
                    float a = m[17] / pl;
                    for (int q = 0; q < 6; ++q) o[q] *= a;
                }
                for (int q = 0; q < 9; ++q) out[(long long)q * g.nc + c] = use_fb ? m[q] : o[q];
                if (use_fb && nfallback) atomicAdd(nfallback, 1u);
            }
        }
        __syncwarp();
    }
}

// features only (training data / analysis): out [nc][12]
__global__ void k_cl_features(Geo g, MxBase mb, VelIn v, double grav, float *out) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.nc) return;
    int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.nxy);
    float f[12], d;
    cl_features(g, mb, v, i, j, k, f, d);
    for (int q = 0; q < 12; ++q) out[c * 12 + q] = f[q];
}

// 4x4x4 (r^3) Favre box filter of a fine flat mixed-precision state into a coarse C-grid state
// (FP64 full fields) and SGS targets t_ij, h_j (FP32, [Nc][9]).  One thread per coarse cell.
__global__ void k_cl_filter(Geo g, MxBase mb, CF5f st, int r, double *cr, double *crt, double *cru, double *crv,
                            double *crw, float *targets) {
    int Nx = g.nx / r, Ny = g.ny / r, Nz = g.nz / r;
    long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long NC = (long long)Nx * Ny * Nz;
    if (C >= NC) return;
    int I = (int)(C % Nx), J = (int)((C / Nx) % Ny), K = (int)(C / ((long long)Nx * Ny));
    double sr = 0, srt = 0, su[3] = {0, 0, 0}, suu[6] = {0, 0, 0, 0, 0, 0}, sut[3] = {0, 0, 0};
    const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int dk = 0; dk < r; ++dk)
        for (int dj = 0; dj < r; ++dj)
            for (int di = 0; di < r; ++di) {
                int i = I * r + di, j = J * r + dj, k = K * r + dk;
                long long c = cix(g, i, j, k);
                double rho = g.rho0[k] + (double)st.r[c];
                double rt = g.rho0[k] * g.th0[k] + (double)st.t[c];
                double rx0 = g.rho0[k] + 0.5 * ((double)fv(g, st.r, i - 1, j, k) + (double)st.r[c]);
                double rx1 = g.rho0[k] + 0.5 * ((double)st.r[c] + (double)fv(g, st.r, i + 1, j, k));
                double ry0 = g.rho0[k] + 0.5 * ((double)fv(g, st.r, i, j - 1, k) + (double)st.r[c]);
                double ry1 = g.rho0[k] + 0.5 * ((double)st.r[c] + (double)fv(g, st.r, i, j + 1, k));
                auto rzf = [&](int kf) -> double {
                    if (kf == 0) return g.rho0[0] + (double)st.r[cix(g, i, j, 0)];
                    if (kf == g.nz) return g.rho0[g.nz - 1] + (double)st.r[cix(g, i, j, g.nz - 1)];
                    return 0.5 * (g.rho0[kf - 1] + g.rho0[kf]) + 0.5 * ((double)st.r[cix(g, i, j, kf - 1)] + (double)st.r[cix(g, i, j, kf)]);
                };
                double u = 0.5 * ((double)st.u[c] / rx0 + (double)__ldg(st.u + cixw(g, i + 1, j, k)) / rx1);
                double vv = 0.5 * ((double)st.v[c] / ry0 + (double)__ldg(st.v + cixw(g, i, j + 1, k)) / ry1);
                double w = 0.5 * ((double)st.w[cix(g, i, j, k)] / rzf(k) + (double)st.w[cix(g, i, j, k + 1)] / rzf(k + 1));
                double th = rt / rho;
                double vel[3] = {u, vv, w};
                sr += rho;
                srt += rt;
                for (int q = 0; q < 3; ++q) { su[q] += rho * vel[q]; sut[q] += rho * vel[q] * th; }
                for (int q = 0; q < 6; ++q) suu[q] += rho * vel[pr[q][0]] * vel[pr[q][1]];
            }
    double n3 = (double)r * r * r;
    double rb = sr / n3;
    double ut[3] = {su[0] / n3 / rb, su[1] / n3 / rb, su[2] / n3 / rb};
    double tht = srt / n3 / rb;
    long long Cc = C;
    cr[Cc] = rb;
    crt[Cc] = srt / n3;
    for (int q = 0; q < 6; ++q) targets[Cc * 9 + q] = (float)(suu[q] / n3 / rb - ut[pr[q][0]] * ut[pr[q][1]]);
    for (int q = 0; q < 3; ++q) targets[Cc * 9 + 6 + q] = (float)(sut[q] / n3 / rb - ut[q] * tht);
    // coarse face momenta: means over the r x r fine faces on each coarse face
    double fu = 0, fvv = 0;
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            fu += (double)st.u[cix(g, I * r, J * r + b, K * r + a)];
            fvv += (double)st.v[cix(g, I * r + b, J * r, K * r + a)];
        }
    cru[Cc] = fu / (r * r);
    crv[Cc] = fvv / (r * r);
    double fw = 0;
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) fw += (double)st.w[cix(g, I * r + b, J * r + a, K * r)];
    crw[Cc] = fw / (r * r);
    if (K == Nz - 1) {   // top coarse w-face row
        long long Ct = ((long long)Nz * Ny + J) * Nx + I;
        double ft = 0;
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) ft += (double)st.w[cix(g, I * r + b, J * r + a, g.nz)];
        crw[Ct] = ft / (r * r);
    }
}

void cl_prepare(const float *d_blob, void *w_bf16, float *b, float *stats, cudaStream_t s) {
    k_cl_prepare<<<(64 * 64 + 255) / 256, 256, 0, s>>>(d_blob, (__nv_bfloat16 *)w_bf16, b, stats);
}
void cl_infer(const Geo &g, const MxBase &mb, const Phys &ph, const void *w_bf16, const float *b,
              const float *stats, const float *ux, const float *vy, const float *wz, const float *thp,
              const float *dr, float *out, unsigned *nfb, cudaStream_t s) {
    const __nv_bfloat16 *w = (const __nv_bfloat16 *)w_bf16;
    ClDev cl{w, w + 1024, w + 1024 + 4096, w + 1024 + 8192, b, stats};
    // persistent grid: as many resident blocks as fit on the device, each looping over tiles
    static int dev_blocks = 0;
    if (dev_blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cl_infer, CLW * 32, 0);
        dev_blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    long long ntiles = (g.nc + 31) / 32;
    long long need = (ntiles + CLW - 1) / CLW;
    unsigned nblk = (unsigned)(need < dev_blocks ? need : dev_blocks);
    mx_launch("mx_closure_mlp", s, [&] {
        k_cl_infer<<<nblk, CLW * 32, 0, s>>>(g, mb, ph, cl, VelIn{ux, vy, wz, thp}, dr, out, nfb);
    });
}
void cl_features_launch(const Geo &g, const MxBase &mb, double grav, const float *ux, const float *vy,
                        const float *wz, const float *thp, float *out, cudaStream_t s) {
    k_cl_features<<<(unsigned)((g.nc + 255) / 256), 256, 0, s>>>(g, mb, VelIn{ux, vy, wz, thp}, grav, out);
}
void cl_filter_launch(const Geo &g, const MxBase &mb, CF5f st, int r, double *cr, double *crt, double *cru,
                      double *crv, double *crw, float *targets, cudaStream_t s) {
    long long NC = (long long)(g.nx / r) * (g.ny / r) * (g.nz / r);
    k_cl_filter<<<(unsigned)((NC + 127) / 128), 128, 0, s>>>(g, mb, st, r, cr, crt, cru, crv, crw, targets);
}

}  // namespace erfk
