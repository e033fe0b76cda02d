// Training kernels of the learned subgrid closure (FP32 master weights, deterministic order).
//
// Network 12 -> 64 -> 64 -> 64 -> 9, SiLU on the hidden layers, MSE on standardised outputs,
// Adam (Kingma & Ba 2015).  Each layer product is a tiled FP32 GEMM with a fixed summation
// order, so a run is reproducible bit for bit.  Parameter layout (FP32, 9737 values):
//   W1[64][12] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[9][64] b4[9]
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/erf.h"
#include "erf_closure.h"

namespace erfk {

// C[M][N] (+)= sum_k A(m,k) B(k,n); A(m,k) = ta ? A[k lda + m] : A[m lda + k], B likewise.
constexpr int TS = 16;
__global__ void k_sgemm(int M, int N, int K, const float *A, int lda, int ta, const float *B, int ldb, int tb,
                        float *C, int ldc, int accumulate) {
    __shared__ float As[TS][TS + 1], Bs[TS][TS + 1];
    int tx = threadIdx.x, ty = threadIdx.y;
    int m = blockIdx.y * TS + ty, n = blockIdx.x * TS + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TS) {
        int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (m < M && ka < K) ? (ta ? A[(long long)ka * lda + m] : A[(long long)m * lda + ka]) : 0.f;
        Bs[ty][tx] = (kb < K && n < N) ? (tb ? B[(long long)n * ldb + kb] : B[(long long)kb * ldb + n]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TS; ++q) acc = fmaf(As[ty][q], Bs[q][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        float *c = C + (long long)m * ldc + n;
        *c = accumulate ? *c + acc : acc;
    }
}

__device__ __forceinline__ float silu_f(float x) { return x / (1.f + expf(-x)); }
__device__ __forceinline__ float dsilu_f(float x) {
    float s = 1.f / (1.f + expf(-x));
    return s * (1.f + x * (1.f - s));
}

// Z += b (per column); A = silu(Z) when act
__global__ void k_bias_act(float *Z, float *A, const float *b, long long rows, int cols, int act) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= rows * cols) return;
    int c = (int)(t % cols);
    float z = Z[t] + b[c];
    Z[t] = z;
    if (act) A[t] = silu_f(z);
}
// G *= dsilu(Z)
__global__ void k_act_back(float *G, const float *Z, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) G[t] *= dsilu_f(Z[t]);
}
// Column reductions, one CTA of CS_T threads per column: thread q sums rows q, q + CS_T, ... in
// order, then a fixed binary tree over the threads; the order is fixed, so the result is
// reproducible bit for bit.
constexpr int CS_T = 256;
template <class T>
__device__ __forceinline__ T cta_tree_sum(T v, T *sh) {
    const int q = threadIdx.x;
    sh[q] = v;
    __syncthreads();
    for (int w = CS_T / 2; w > 0; w >>= 1) {
        if (q < w) sh[q] += sh[q + w];
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();   // sh may be reused at once
    return r;
}
// out[c] = sum over rows of G[r][c]
__global__ void __launch_bounds__(CS_T) k_colsum(const float *G, long long rows, int cols, float *out) {
    __shared__ float sh[CS_T];
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < rows; r += CS_T) s += G[r * cols + c];
    s = cta_tree_sum(s, sh);
    if (threadIdx.x == 0) out[c] = s;
}
// dY = 2 (Y - T) / (rows cols); per-block partial sums of (Y - T)^2
__global__ void k_mse(const float *Y, const float *T, float *dY, long long n, float scale, float *part) {
    __shared__ float sm[256];
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float e = 0.f;
    if (t < n) {
        float d = Y[t] - T[t];
        dY[t] = 2.f * d * scale;
        e = d * d;
    }
    sm[threadIdx.x] = e;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_loss_final(const float *part, int nparts, float scale, float *loss) {
    if (threadIdx.x || blockIdx.x) return;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += part[b];
    *loss = s * scale;
}
__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float gt = g[t];
    float mt = b1 * m[t] + (1.f - b1) * gt;
    float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}
// column mean / standard deviation over rows (FP64 accumulation, one CTA per column)
__global__ void __launch_bounds__(CS_T) k_col_stats(const float *A, long long rows, int cols, float *mean, float *sd) {
    __shared__ double sh[CS_T];
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (long long r = threadIdx.x; r < rows; r += CS_T) {
        double x = A[r * cols + c];
        s += x;
        s2 += x * x;
    }
    s = cta_tree_sum(s, sh);
    s2 = cta_tree_sum(s2, sh);
    if (threadIdx.x != 0) return;
    double mu = s / (double)rows;
    double var = s2 / (double)rows - mu * mu;
    double d = var > 0.0 ? sqrt(var) : 0.0;
    mean[c] = (float)mu;
    sd[c] = d > 0.0 ? (float)d : 1.f;
}
__global__ void k_standardise(const float *A, float *out, long long rows, int cols, const float *mean,
                              const float *sd) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= rows * cols) return;
    int c = (int)(t % cols);
    out[t] = (A[t] - mean[c]) / sd[c];
}

namespace {
inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
void gemm(int M, int N, int K, const float *A, int lda, int ta, const float *B, int ldb, int tb, float *C, int ldc,
          int acc, cudaStream_t s) {
    dim3 blk(TS, TS), grd((N + TS - 1) / TS, (M + TS - 1) / TS);
    k_sgemm<<<grd, blk, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, acc);
}
struct Views {
    float *W[4], *b[4];
};
Views views(float *p) {
    Views v;
    const int in[4] = {CL_NIN, CL_NH, CL_NH, CL_NH}, out[4] = {CL_NH, CL_NH, CL_NH, CL_NOUT};
    float *q = p;
    for (int l = 0; l < 4; ++l) {
        v.W[l] = q;
        q += in[l] * out[l];
        v.b[l] = q;
        q += out[l];
    }
    return v;
}
}  // namespace

size_t train_scratch_floats(int batch) {
    // activations Z1..Z3, A1..A3 (6 x B x 64), Y, dY (2 x B x 9), G (2 x B x 64), grads, m, v, loss parts
    return (size_t)batch * (6 * CL_NH + 2 * CL_NOUT + 2 * CL_NH) + 3 * (size_t)CL_NPARAM + nb((long long)batch * CL_NOUT, 256) + 16;
}

// forward + backward of one batch: loss into *d_loss, gradients into g (overwritten)
static void fwd_bwd(const float *X, const float *T, int B, float *p, float *g, float *S, float *d_loss,
                    cudaStream_t s) {
    const int H = CL_NH, O = CL_NOUT, I = CL_NIN;
    Views P = views(p), Gv = views(g);
    float *Z[3], *A[3];
    for (int l = 0; l < 3; ++l) {
        Z[l] = S + (size_t)(2 * l) * B * H;
        A[l] = S + (size_t)(2 * l + 1) * B * H;
    }
    float *Y = S + (size_t)6 * B * H, *dY = Y + (size_t)B * O;
    float *G0 = dY + (size_t)B * O, *G1 = G0 + (size_t)B * H;
    float *part = G1 + (size_t)B * H + 3 * (size_t)CL_NPARAM;
    // forward
    const float *in = X;
    int nin = I;
    for (int l = 0; l < 3; ++l) {
        gemm(B, H, nin, in, nin, 0, P.W[l], nin, 1, Z[l], H, 0, s);
        k_bias_act<<<nb((long long)B * H, 256), 256, 0, s>>>(Z[l], A[l], P.b[l], B, H, 1);
        in = A[l];
        nin = H;
    }
    gemm(B, O, H, A[2], H, 0, P.W[3], H, 1, Y, O, 0, s);
    k_bias_act<<<nb((long long)B * O, 256), 256, 0, s>>>(Y, nullptr, P.b[3], B, O, 0);
    long long ny = (long long)B * O;
    unsigned np = nb(ny, 256);
    k_mse<<<np, 256, 0, s>>>(Y, T, dY, ny, 1.f / (float)ny, part);
    k_loss_final<<<1, 32, 0, s>>>(part, (int)np, 1.f / (float)ny, d_loss);
    // backward: layer 4
    gemm(O, H, B, dY, O, 1, A[2], H, 0, Gv.W[3], H, 0, s);
    k_colsum<<<O, CS_T, 0, s>>>(dY, B, O, Gv.b[3]);
    gemm(B, H, O, dY, O, 0, P.W[3], H, 0, G0, H, 0, s);
    float *gcur = G0, *gnext = G1;
    for (int l = 2; l >= 0; --l) {
        k_act_back<<<nb((long long)B * H, 256), 256, 0, s>>>(gcur, Z[l], (long long)B * H);
        const float *a_in = l == 0 ? X : A[l - 1];
        int nin_l = l == 0 ? I : H;
        gemm(H, nin_l, B, gcur, H, 1, a_in, nin_l, 0, Gv.W[l], nin_l, 0, s);
        k_colsum<<<H, CS_T, 0, s>>>(gcur, B, H, Gv.b[l]);
        if (l > 0) {
            gemm(B, H, H, gcur, H, 0, P.W[l], H, 0, gnext, H, 0, s);
            float *t = gcur; gcur = gnext; gnext = t;
        }
    }
}

}  // namespace erfk

using namespace erfk;

extern "C" size_t erf_train_scratch_bytes(int32_t batch) {
    return batch > 0 ? train_scratch_floats(batch) * sizeof(float) : 0;
}

extern "C" erf_status erf_closure_grad(const float *d_X, const float *d_T, int32_t n, float *d_params,
                                       float *d_grad, float *d_loss, void *d_scratch, size_t scratch_bytes,
                                       void *cuda_stream) {
    if (!d_X || !d_T || !d_params || !d_grad || !d_loss || !d_scratch || n < 1) return ERF_EINVAL;
    if (scratch_bytes < erf_train_scratch_bytes(n)) return ERF_ENOSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    fwd_bwd(d_X, d_T, n, d_params, d_grad, (float *)d_scratch, d_loss, s);
    return cudaGetLastError() == cudaSuccess ? ERF_OK : ERF_ECUDA;
}

extern "C" erf_status erf_train_closure(const erf_train_cfg *cfg, const float *d_X, const float *d_T, int64_t n,
                                        float *d_params, float *d_losses, void *d_scratch, size_t scratch_bytes,
                                        void *cuda_stream) {
    if (!cfg || !d_X || !d_T || !d_params || !d_scratch || n < 1 || cfg->batch < 1 || cfg->epochs < 0) return ERF_EINVAL;
    if (scratch_bytes < erf_train_scratch_bytes(cfg->batch)) return ERF_ENOSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    float *S = (float *)d_scratch;
    const int B = cfg->batch;
    float *grad = S + (size_t)B * (6 * CL_NH + 2 * CL_NOUT + 2 * CL_NH);
    float *m = grad + CL_NPARAM, *v = m + CL_NPARAM;
    cudaMemsetAsync(m, 0, 2 * CL_NPARAM * sizeof(float), s);
    long long t = 0;
    for (int ep = 0; ep < cfg->epochs; ++ep)
        for (long long s0 = 0; s0 < n; s0 += B) {
            int bsz = (int)((n - s0) < B ? (n - s0) : B);
            float *loss = d_losses ? d_losses + t : grad + 3 * CL_NPARAM;   // scratch word when not recorded
            fwd_bwd(d_X + s0 * CL_NIN, d_T + s0 * CL_NOUT, bsz, d_params, grad, S, loss, s);
            ++t;
            float c1 = 1.f - powf(cfg->beta1, (float)t), c2 = 1.f - powf(cfg->beta2, (float)t);
            k_adam<<<nb(CL_NPARAM, 256), 256, 0, s>>>(d_params, grad, m, v, CL_NPARAM, cfg->lr, cfg->beta1, cfg->beta2,
                                                      cfg->eps, c1, c2);
        }
    return cudaGetLastError() == cudaSuccess ? ERF_OK : ERF_ECUDA;
}

extern "C" erf_status erf_column_stats(const float *d_A, int64_t rows, int32_t cols, float *d_mean, float *d_std,
                                       void *cuda_stream) {
    if (!d_A || !d_mean || !d_std || rows < 1 || cols < 1) return ERF_EINVAL;
    k_col_stats<<<cols, CS_T, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(d_A, rows, cols, d_mean, d_std);
    return cudaGetLastError() == cudaSuccess ? ERF_OK : ERF_ECUDA;
}

extern "C" erf_status erf_standardise(const float *d_A, int64_t rows, int32_t cols, const float *d_mean,
                                      const float *d_std, float *d_out, void *cuda_stream) {
    if (!d_A || !d_mean || !d_std || !d_out || rows < 1 || cols < 1) return ERF_EINVAL;
    k_standardise<<<nb(rows * cols, 256), 256, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(d_A, d_out, rows, cols,
                                                                                                d_mean, d_std);
    return cudaGetLastError() == cudaSuccess ? ERF_OK : ERF_ECUDA;
}
