// Advection interpolants shared by the FP64 and the mixed-precision kernels (Sec. 3.6).
#pragma once
#include <cuda_runtime.h>

namespace erfk {

// q[0..5] = q_{m-3}..q_{m+2}; 5th-order upwind value at m-1/2 for s = sign of the advecting
// normal momentum there.  The centred sixth-order value minus s/60 times its dissipative part
// (Sec. 3.6) is, for s = +1 and -1, the five-point stencil (2, -13, 47, 27, -3)/60 over the five
// points on the upwind side: the side is selected (no FP64 work) and the stencil takes five
// multiply-adds instead of thirteen operations.  s = 0 takes the left side; every caller
// multiplies the value by that zero momentum.
template <class T>
__device__ __forceinline__ T upwind5(const T *q, T s) {
    const bool l = s >= T(0);
    const T a0 = l ? q[0] : q[5], a1 = l ? q[1] : q[4], a2 = l ? q[2] : q[3], a3 = l ? q[3] : q[2];
    const T a4 = l ? q[4] : q[1];
    return fma(T(47.0 / 60.0), a2, fma(T(27.0 / 60.0), a3, fma(T(-13.0 / 60.0), a1,
               fma(T(2.0 / 60.0), a0, T(-3.0 / 60.0) * a4))));
}
template <class T>
__device__ __forceinline__ T sgnT(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0)); }

// WENO5-JS (Jiang & Shu 1996) or WENO5-Z (Borges et al. 2008) face value; upwind side s >= 0
// is the left.  The nonlinear weights are normalised with one division.
template <class T>
__device__ __forceinline__ T weno5(const T *q, T s, int zflag) {
    T a, b, c, d, e;   // v_{-2}, v_{-1}, v_0, v_1, v_2 on the upwind side
    if (s >= T(0)) { a = q[0]; b = q[1]; c = q[2]; d = q[3]; e = q[4]; }
    else { a = q[5]; b = q[4]; c = q[3]; d = q[2]; e = q[1]; }
    const T eps = T(1.0e-6);
    T p0 = (T(2) * a - T(7) * b + T(11) * c) * T(1.0 / 6.0);
    T p1 = (-b + T(5) * c + T(2) * d) * T(1.0 / 6.0);
    T p2 = (T(2) * c + T(5) * d - e) * T(1.0 / 6.0);
    T t0 = a - T(2) * b + c, u0 = a - T(4) * b + T(3) * c;
    T t1 = b - T(2) * c + d, u1 = b - d;
    T t2 = c - T(2) * d + e, u2 = T(3) * c - T(4) * d + e;
    T b0 = T(13.0 / 12.0) * t0 * t0 + T(0.25) * u0 * u0;
    T b1 = T(13.0 / 12.0) * t1 * t1 + T(0.25) * u1 * u1;
    T b2 = T(13.0 / 12.0) * t2 * t2 + T(0.25) * u2 * u2;
    T w0, w1, w2;
    if (zflag) {
        // alpha_k = d_k (1 + tau/(b_k + eps)) scaled by prod (b_j + eps)
        T tau = fabs(b0 - b2);
        T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
        w0 = T(0.1) * (e0 + tau) * e1 * e2;
        w1 = T(0.6) * (e1 + tau) * e0 * e2;
        w2 = T(0.3) * (e2 + tau) * e0 * e1;
    } else {
        // alpha_k = d_k / (eps + b_k)^2 scaled by prod (eps + b_j)^2
        T e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
        T f01 = e0 * e1, f02 = e0 * e2, f12 = e1 * e2;
        w0 = T(0.1) * f12 * f12;
        w1 = T(0.6) * f02 * f02;
        w2 = T(0.3) * f01 * f01;
    }
    return (w0 * p0 + w1 * p1 + w2 * p2) / (w0 + w1 + w2);
}

}  // namespace erfk
