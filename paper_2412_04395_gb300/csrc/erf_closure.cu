// Learned subgrid closure: features, BF16 tensor-core inference with Smagorinsky fallback, the
// 4x box filter that makes training targets, and the weight upload.
//
// Inference maps each cell's 12 features (resolved velocity gradients, dtheta/dx, dtheta/dy, N^2)
// through 12 -> 64 -> 64 -> 64 -> 9 (SiLU) to the kinematic SGS stress and heat flux on the
// fifth-generation tensor cores (tcgen05).  A CTA of 128 threads takes 128-cell tiles, one cell
// per thread: the thread writes its cell's standardised features (BF16) as row t of the
// activation operand in shared memory; one elected thread issues each layer as M = 128 x N = 64
// (output layer N = 16) MMAs with K = 16 steps into a TMEM accumulator; every thread then reads
// its own row back (TMEM lane t), adds the bias, applies SiLU and writes the BF16 activations
// as the next layer's operand.  The weights stay in shared memory for the CTA's lifetime, and
// each layer's completion is an mbarrier that the MMAs' commit arrives on (bounded waits).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/erf.h"
#include "erf_closure.h"
#include "erf_dev.cuh"
#include "erf_launch.h"
#include "erf_mixed.h"
#include "erf_tc.cuh"

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
// SiLU of x = acc + b as h (1 + tanh h), h = x/2 = fma(acc, 1/2, b/2) (hb = b/2): one MUFU
// operation (tanh.approx.f32, relative error about 2^-11) instead of an exponential and a
// reciprocal.  The activation is rounded to BF16 (2^-9) right after, and the inference error
// against a BF16-emulating FP64 network stays at 2e-5 .. 2e-4 relative L2 (measured; the test
// bound is 5e-3).
__device__ __forceinline__ float silu_half(float acc, float hb) {
    float h = fmaf(acc, 0.5f, hb), t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// Learned SGS stress/heat flux at every cell (mixed path), with Smagorinsky as the per-cell
// fallback and backscatter limited to half the Smagorinsky transfer.  Persistent CTAs of 128
// threads load the weights once into the canonical K-major operand layout and loop over 128-cell
// tiles.  Every wait on an MMA barrier is bounded: a CTA whose wait gives up sets bit 2 of *err,
// waits once more (bounded) for its MMAs, frees its TMEM and stops.
// out: 9 planes of nc floats: rho t11, rho t22, rho t33, rho t12, rho t13, rho t23, rho h1..h3.
constexpr int CLT = 128;            // threads per CTA = cells per tile = MMA rows
constexpr int CL_NM = 18;           // per-cell values the output step needs (fallback, strain, bound)

// Step 1 of a tile: cell c's standardised features (BF16) into its row of the activation
// operand; the Smagorinsky fallback stresses m[0..8], the density m[9], the strain m[11..16] and
// the backscatter bound m[17]; fb = 1 if a feature lies outside the training range (|z| > 6).
__device__ __forceinline__ void cl_cell_inputs(const Geo &g, const MxBase &mb, const VelIn &v, const float *dr,
                                               const float *in_mu, const float *in_rsd, float rPr, long long c,
                                               bool valid, unsigned char *row, float *m, int &fb) {
    float z[12];
    for (int q = 0; q < 12; ++q) z[q] = 0.f;
    for (int q = 0; q < CL_NM; ++q) m[q] = 0.f;
    fb = 0;
    if (valid) {
        unsigned rw = (unsigned)(c / g.nx);
        int i = (int)(c - (long long)rw * g.nx);
        int j = (int)(rw % (unsigned)g.ny), k = (int)(rw / (unsigned)g.ny);
        float f[12], dthdz;
        cl_features(g, mb, v, i, j, k, f, dthdz);
        for (int q = 0; q < 12; ++q) {
            z[q] = (f[q] - in_mu[q]) * in_rsd[q];
            if (!(fabsf(z[q]) <= 6.f)) fb = 1;
        }
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
        // backscatter bound: the learned transfer -t_ij S_ij may not fall below -1/2 of the
        // Smagorinsky transfer (both density-weighted)
        float ps = -(m[0] * s11 + m[1] * s22 + m[2] * s33 + 2.f * (m[3] * s12 + m[4] * s13 + m[5] * s23));
        m[17] = -0.5f * ps;
    }
    *reinterpret_cast<uint4 *>(row) =
        make_uint4(pack_bf16(z[0], z[1]), pack_bf16(z[2], z[3]), pack_bf16(z[4], z[5]), pack_bf16(z[6], z[7]));
    *reinterpret_cast<uint4 *>(row + 128) = make_uint4(pack_bf16(z[8], z[9]), pack_bf16(z[10], z[11]), 0u, 0u);
}

// Step 2: this thread's accumulator row of a hidden layer (64 FP32 columns of TMEM) + bias,
// SiLU, back into its operand row as BF16 (hb: the layer's half biases)
__device__ __forceinline__ void cl_row_silu(uint32_t tlane, const float *hb, unsigned char *row) {
    for (int h = 0; h < 2; ++h) {
        uint32_t r[32];
        tc_ld32(tlane + 32u * h, r);
        uint32_t pk[16];
        for (int q = 0; q < 16; ++q)
            pk[q] = pack_bf16(silu_half(__uint_as_float(r[2 * q]), hb[32 * h + 2 * q]),
                              silu_half(__uint_as_float(r[2 * q + 1]), hb[32 * h + 2 * q + 1]));
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<uint4 *>(row + (4 * h + u) * 128) =
                make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
    }
}

// Step 3: the output row (9 of 16 columns), de-standardised, density-weighted, bounded, or the
// fallback; stored to the 9 planes
__device__ __forceinline__ void cl_cell_output(uint32_t tlane, const float *sb4, const float *out_mu,
                                               const float *out_sd, const float *m, int fb, bool valid,
                                               long long c, long long nc, float *out, unsigned *nfallback) {
    uint32_t r[16];
    tc_ld16(tlane, r);
    if (!valid) return;
    int use_fb = fb;
    float o[9];
    for (int q = 0; q < 9; ++q) {
        o[q] = (__uint_as_float(r[q]) + sb4[q]) * out_sd[q] + out_mu[q];
        if (!isfinite(o[q])) use_fb = 1;
    }
    float rho = m[9];
    for (int q = 0; q < 9; ++q) o[q] *= rho;
    float pl = -(o[0] * m[11] + o[1] * m[12] + o[2] * m[13] + 2.f * (o[3] * m[14] + o[4] * m[15] + o[5] * m[16]));
    if (pl < m[17]) {
        float a = m[17] / pl;
        for (int q = 0; q < 6; ++q) o[q] *= a;
    }
    for (int q = 0; q < 9; ++q) out[(long long)q * nc + c] = use_fb ? m[q] : o[q];
    if (use_fb && nfallback) atomicAdd(nfallback, 1u);
}

// the MMAs of layer L (0: K = 16 -> N = 64; 1, 2: K = 64 -> N = 64; 3: K = 64 -> N = 16) of the
// tile whose operand is dA into the accumulator at TMEM address tm; issued by one thread
struct ClDesc {
    uint64_t W1, W2, W3, W4;
};
__device__ __forceinline__ void cl_issue_layer(int layer, uint32_t tm, uint64_t dA, const ClDesc &dw) {
    constexpr uint32_t I64 = tc_idesc_bf16(128, 64), I16 = tc_idesc_bf16(128, 16);
    if (layer == 0) {
        tc_mma_bf16(tm, dA, dw.W1, I64, 0u);
    } else {
        const uint64_t dW = layer == 1 ? dw.W2 : (layer == 2 ? dw.W3 : dw.W4);
        const uint32_t id = layer == 3 ? I16 : I64;
        for (int s = 0; s < 4; ++s) tc_mma_bf16(tm, dA + 16u * s, dW + 16u * s, id, s > 0 ? 1u : 0u);
    }
}

// One tile per pass: 128 threads, 64 TMEM columns and 38 KB of static shared memory per CTA,
// five CTAs per SM.  Measured and not kept: two tiles in flight per CTA (while the tensor cores run
// one tile's layer the threads run the other's SiLU; three CTAs per SM for its 73 KB of shared
// memory) took 200 ms per step at 2048^2 x 160 against 141 ms; the kernel is bound by its SIMT
// work's issue and latency at the warps an SM holds, not by the MMA round trips.
constexpr uint32_t CL_TCOLS = 64;
constexpr int CL_CTAS_PER_SM = 5;
__global__ void __launch_bounds__(CLT, CL_CTAS_PER_SM) k_cl_infer(Geo g, MxBase mb, Phys ph, ClDev cl, VelIn v,
                                                                    const float *dr, float *out, unsigned *nfallback,
                                                                    unsigned *err) {
    __shared__ __align__(1024) unsigned char sA[128 * 64 * 2];
    __shared__ __align__(1024) unsigned char sW1[64 * 16 * 2];
    __shared__ __align__(1024) unsigned char sW2[64 * 64 * 2];
    __shared__ __align__(1024) unsigned char sW3[64 * 64 * 2];
    __shared__ __align__(1024) unsigned char sW4[16 * 64 * 2];
    __shared__ float shb[3 * 64];
    __shared__ float sb4[16];
    __shared__ float sst[2 * CL_NIN + 2 * CL_NOUT];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x, warp = t >> 5;
    auto put = [&](unsigned char *dst, const __nv_bfloat16 *src, int rows, int K) {
        for (int q = t; q < rows * K; q += CLT) *reinterpret_cast<__nv_bfloat16 *>(dst + tc_off(q / K, q % K, K)) = src[q];
    };
    put(sW1, cl.W1, 64, 16);
    put(sW2, cl.W2, 64, 64);
    put(sW3, cl.W3, 64, 64);
    put(sW4, cl.W4, 16, 64);
    for (int q = t; q < 192; q += CLT) shb[q] = 0.5f * cl.b[q];
    if (t < 16) sb4[t] = cl.b[192 + t];
    if (t < 2 * CL_NIN + 2 * CL_NOUT) sst[t] = (t >= CL_NIN && t < 2 * CL_NIN) ? 1.f / cl.stats[t] : cl.stats[t];
    if (t == 0) mbar_init(&bar, 1);
    if (warp == 0) {
        tc_alloc(&s_taddr, CL_TCOLS);
        tc_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s_taddr, tlane = tm + ((uint32_t)(32 * warp) << 16);
    const uint64_t dA = tc_smem_desc(smem_u32(sA), 128, 1024);
    const ClDesc dw{tc_smem_desc(smem_u32(sW1), 128, 256), tc_smem_desc(smem_u32(sW2), 128, 1024),
                    tc_smem_desc(smem_u32(sW3), 128, 1024), tc_smem_desc(smem_u32(sW4), 128, 1024)};
    const float *in_mu = sst, *in_rsd = sst + 12, *out_mu = sst + 24, *out_sd = sst + 33;
    unsigned char *row = sA + (t >> 3) * 1024 + (t & 7) * 16;
    unsigned phase = 0, pend = 0;
    int timeout = 0, aborted = 0;
    auto sync_layer = [&]() -> int {
        fence_async_smem();
        tc_fence_before();
        int ab = __syncthreads_or(timeout);
        tc_fence_after();
        return ab;
    };
    auto run_layer = [&](int layer) {
        if (t == 0) {
            cl_issue_layer(layer, tm, dA, dw);
            tc_commit(&bar);
        }
        pend = phase;
        if (!mbar_wait_bounded(&bar, phase, TMA_MAX_POLLS)) timeout = 1;
        phase ^= 1u;
        tc_fence_after();
    };
    const long long ntiles = (g.nc + CLT - 1) / CLT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long c = tile * CLT + t;
        const bool valid = c < g.nc;
        float m[CL_NM];
        int fb;
        cl_cell_inputs(g, mb, v, dr, in_mu, in_rsd, mb.rPr, c, valid, row, m, fb);
        for (int layer = 0; layer < 3 && !aborted; ++layer) {
            if (sync_layer()) { aborted = 1; break; }
            run_layer(layer);
            cl_row_silu(tlane, shb + 64 * layer, row);
        }
        if (aborted || sync_layer()) { aborted = 1; break; }
        run_layer(3);
        cl_cell_output(tlane, sb4, out_mu, out_sd, m, fb, valid, c, g.nc, out, nfallback);
    }
    tc_fence_before();
    if (__syncthreads_or(timeout) || aborted) {
        if (t == 0 && err) atomicOr(err, 2u);
        mbar_wait_bounded(&bar, pend, TMA_MAX_POLLS);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tm, CL_TCOLS);
}


// Self-test of the tensor-core path on exact integer data: the operand shapes of the network
// (K = 64 with N = 64 and with N = 16; K = 16 with N = 64) through the same descriptors and
// layouts, compared with the products formed by plain integer loops.  mism counts mismatching
// outputs; bit 0 of *flag reports a wait that gave up.
constexpr int TCS_SMEM = 64 * 1024;   // generous: three operands need 26 KB
__global__ void __launch_bounds__(128, 1) k_tc_selftest(int *mism, unsigned *flag) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x, warp = t >> 5;
    unsigned char *sA = dsm, *sB = dsm + 16384, *sB1 = dsm + 24576;   // A [128][64], B [64][64], B1 [64][16]
    auto av = [](int m, int k) { return ((m * 7 + k * 3) % 9) - 4; };
    auto bv = [](int n, int k) { return ((n * 5 + k * 11) % 7) - 3; };
    for (int q = t; q < 128 * 64; q += 128)
        *reinterpret_cast<__nv_bfloat16 *>(sA + tc_off(q / 64, q % 64, 64)) = __float2bfloat16_rn((float)av(q / 64, q % 64));
    for (int q = t; q < 64 * 64; q += 128)
        *reinterpret_cast<__nv_bfloat16 *>(sB + tc_off(q / 64, q % 64, 64)) = __float2bfloat16_rn((float)bv(q / 64, q % 64));
    for (int q = t; q < 64 * 16; q += 128)
        *reinterpret_cast<__nv_bfloat16 *>(sB1 + tc_off(q / 16, q % 16, 16)) = __float2bfloat16_rn((float)bv(q / 16, q % 16));
    if (t == 0) mbar_init(&bar, 1);
    if (warp == 0) {
        tc_alloc(&s_taddr, 256);
        tc_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s_taddr;
    if (t == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), b1 = smem_u32(sB1);
        for (int s = 0; s < 4; ++s)   // K = 64, N = 64 -> columns 0..63
            tc_mma_bf16(tm, tc_smem_desc(a0 + 256 * s, 128, 1024), tc_smem_desc(b0 + 256 * s, 128, 1024),
                        tc_idesc_bf16(128, 64), s > 0 ? 1u : 0u);
        for (int s = 0; s < 4; ++s)   // K = 64, N = 16 (rows 0..15 of B) -> columns 64..79
            tc_mma_bf16(tm + 64, tc_smem_desc(a0 + 256 * s, 128, 1024), tc_smem_desc(b0 + 256 * s, 128, 1024),
                        tc_idesc_bf16(128, 16), s > 0 ? 1u : 0u);
        // K = 16 (columns 0..15 of A, in its K = 64 layout), N = 64 from B1 -> columns 128..191
        tc_mma_bf16(tm + 128, tc_smem_desc(a0, 128, 1024), tc_smem_desc(b1, 128, 256), tc_idesc_bf16(128, 64), 0u);
        tc_commit(&bar);
    }
    int to = mbar_wait_bounded(&bar, 0, TMA_MAX_POLLS) ? 0 : 1;
    tc_fence_after();
    if (__syncthreads_or(to)) {
        if (t == 0) atomicOr(flag, 1u);
        mbar_wait_bounded(&bar, 0, TMA_MAX_POLLS);
    } else {
        const uint32_t lane = tm + ((uint32_t)(32 * warp) << 16);
        const int mr = t;   // TMEM lane = row of D
        int bad = 0;
        uint32_t r[32];
        for (int h = 0; h < 2; ++h) {
            tc_ld32(lane + 32u * h, r);
            for (int q = 0; q < 32; ++q) {
                int n = 32 * h + q, e = 0;
                for (int k = 0; k < 64; ++k) e += av(mr, k) * bv(n, k);
                bad += __uint_as_float(r[q]) != (float)e;
            }
        }
        tc_ld16(lane + 64u, r);
        for (int n = 0; n < 16; ++n) {
            int e = 0;
            for (int k = 0; k < 64; ++k) e += av(mr, k) * bv(n, k);
            bad += __uint_as_float(r[n]) != (float)e;
        }
        for (int h = 0; h < 2; ++h) {
            tc_ld32(lane + 128u + 32u * h, r);
            for (int q = 0; q < 32; ++q) {
                int n = 32 * h + q, e = 0;
                for (int k = 0; k < 16; ++k) e += av(mr, k) * bv(n, k);
                bad += __uint_as_float(r[q]) != (float)e;
            }
        }
        if (bad) atomicAdd(mism, bad);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tm, 256);
}
void selftest_tensor_cores(int *mism, unsigned *flag, cudaStream_t s) {
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, TCS_SMEM);
    k_tc_selftest<<<1, 128, TCS_SMEM, s>>>(mism, flag);
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
              const float *dr, float *out, unsigned *nfb, unsigned *err, cudaStream_t s) {
    const __nv_bfloat16 *w = (const __nv_bfloat16 *)w_bf16;
    ClDev cl{w, w + 1024, w + 1024 + 4096, w + 1024 + 8192, b, stats};
    // persistent grid: CL_CTAS_PER_SM CTAs per SM, the residency the launch bounds guarantee for
    // registers (at most 102 per thread for 5 CTAs) and that the 38 KB of shared memory allows
    // (5 x 39 KB of the SM's 228 KB; 6 would not fit).  (The runtime's occupancy query reports one
    // block per SM for kernels that allocate TMEM.)  Their TMEM, 64 columns each, fits the SM's
    // 512.  Measured at 2048^2 x 160: 5 CTAs per SM 5% faster than 4.
    static_assert(CL_CTAS_PER_SM * CL_TCOLS <= 512, "TMEM of the resident CTAs exceeds an SM's 512 columns");
    static int dev_blocks = 0;
    if (dev_blocks == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dev_blocks = sms * CL_CTAS_PER_SM;
    }
    long long ntiles = (g.nc + CLT - 1) / CLT;
    unsigned nblk = (unsigned)(ntiles < dev_blocks ? ntiles : dev_blocks);
    mx_launch("mx_closure_mlp", s, [&] {
        k_cl_infer<<<nblk, CLT, 0, s>>>(g, mb, ph, cl, VelIn{ux, vy, wz, thp}, dr, out, nfb, err);
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
