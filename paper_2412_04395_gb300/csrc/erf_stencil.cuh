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
// upwind5_side takes the side itself (l: the left one) and every weight times H; H a power of two
// scales the result exactly (the FP64 momentum fluxes fold the 1/2 of their face average into it).
template <class T, int H = 1>
__device__ __forceinline__ T upwind5_side(const T *q, bool l) {
    constexpr T h = H == 1 ? T(1) : T(0.5);
    const T a0 = l ? q[0] : q[5], a1 = l ? q[1] : q[4], a2 = l ? q[2] : q[3], a3 = l ? q[3] : q[2];
    const T a4 = l ? q[4] : q[1];
    return fma(T(47.0 / 60.0) * h, a2, fma(T(27.0 / 60.0) * h, a3, fma(T(-13.0 / 60.0) * h, a1,
               fma(T(2.0 / 60.0) * h, a0, (T(-3.0 / 60.0) * h) * a4))));
}
template <class T>
__device__ __forceinline__ T upwind5(const T *q, T s) {
    return upwind5_side<T>(q, s >= T(0));
}
// q[0..5] = q_{m-3}..q_{m+2}; 3rd-order upwind value at m-1/2: the centred fourth-order value
// plus s/12 times its dissipative part (Sec. 3.6), i.e. (-1, 5, 2)/6 over the three points on the
// upwind side (s = 0 takes the left side; every caller multiplies by that zero momentum)
template <class T, int H = 1>
__device__ __forceinline__ T upwind3_side(const T *q, bool l) {
    constexpr T h = H == 1 ? T(1) : T(0.5);
    const T a0 = l ? q[1] : q[4], a1 = l ? q[2] : q[3], a2 = l ? q[3] : q[2];
    return fma(T(5.0 / 6.0) * h, a1, fma(T(1.0 / 3.0) * h, a2, (T(-1.0 / 6.0) * h) * a0));
}
template <class T>
__device__ __forceinline__ T upwind3(const T *q, T s) {
    return upwind3_side<T>(q, s >= T(0));
}
// face value of an advected scalar: WENO5-JS (scheme 0), WENO5-Z (1) or upwind-3 (3); defined
// after weno5 below
template <class T>
__device__ __forceinline__ T scal_face(const T *q, T s, int scheme);
// the momentum interpolant of the configuration (upwind-3 or upwind-5)
template <class T>
__device__ __forceinline__ T upwind_mom(const T *q, T s, int mom3) {
    return mom3 ? upwind3(q, s) : upwind5(q, s);
}

template <class T>
__device__ __forceinline__ T sgnT(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0)); }
// correctly rounded reciprocal (FP32: one MUFU operation and its refinement instead of a division)
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

// WENO5-JS (Jiang & Shu 1996) or WENO5-Z (Borges et al. 2008) face value in FP32 (the
// mixed-precision kernels); upwind side s >= 0 is the left.  The three candidates
// p0 = (2a - 7b + 11c)/6, p1 = (-b + 5c + 2d)/6, p2 = (2c + 5d - e)/6 enter as
// p1 + (w0 (p0 - p1) + w2 (p2 - p1)) / sum w, with p0 - p1 = (t0 - t1)/3 and
// p2 - p1 = (t1 - t2)/6 from the indicator terms; the indicators 13/12 t^2 + 1/4 u^2 and
// eps = 1e-6 carry a common factor 12/13 (the weights are homogeneous in eps + beta); the
// normalisation takes one correctly rounded reciprocal.
template <class T>
__device__ __forceinline__ T weno5(const T *q, T s, int zflag) {
    T a, b, c, d, e;   // v_{-2}, v_{-1}, v_0, v_1, v_2 on the upwind side
    if (s >= T(0)) { a = q[0]; b = q[1]; c = q[2]; d = q[3]; e = q[4]; }
    else { a = q[5]; b = q[4]; c = q[3]; d = q[2]; e = q[1]; }
    const T d1 = a - b, d2 = b - c, d3 = c - d, d4 = d - e;
    const T p1 = fma(T(-1.0 / 6.0), d2, fma(T(-1.0 / 3.0), d3, c));
    const T t0 = d1 - d2, u0 = fma(T(-3), d2, d1);
    const T t1 = d2 - d3, u1 = d2 + d3;
    const T t2 = d3 - d4, u2 = fma(T(3), d3, -d4);
    const T q0 = t0 - t1, q2 = t1 - t2;
    // e_r = eps + beta_r (scaled), eps inside the indicator FMAs
    const T k3 = T(3.0 / 13.0), eps = T(1.0e-6 * (12.0 / 13.0));
    const T e0 = fma(t0, t0, fma(k3 * u0, u0, eps));
    const T e1 = fma(t1, t1, fma(k3 * u1, u1, eps));
    const T e2 = fma(t2, t2, fma(k3 * u2, u2, eps));
    T N, D;
    if (zflag) {
        // alpha_k = d_k (1 + tau/(b_k + eps)) scaled by prod (b_j + eps)
        const T tau = fabs(e0 - e2);
        const T w0 = T(0.1) * (e0 + tau) * e1 * e2;
        const T w1 = T(0.6) * (e1 + tau) * e0 * e2;
        const T w2 = T(0.3) * (e2 + tau) * e0 * e1;
        N = fma(w0, T(1.0 / 3.0) * q0, w2 * (T(1.0 / 6.0) * q2));
        D = w0 + w1 + w2;
    } else {
        // alpha_k = d_k / (eps + b_k)^2 scaled by prod (eps + b_j)^2 and by 10/3
        const T f01 = e0 * e1, f02 = e0 * e2, f12 = e1 * e2;
        const T g0 = f12 * f12, g1 = f02 * f02, g2 = f01 * f01;
        D = fma(T(1.0 / 3.0), g0, fma(T(2), g1, g2));
        N = fma(g0 * T(1.0 / 9.0), q0, g2 * (T(1.0 / 6.0) * q2));
    }
    return fma(N, rcp_t(D), p1);
}

template <class T>
__device__ __forceinline__ T scal_face(const T *q, T s, int scheme) {
    return scheme == 3 ? upwind3(q, s) : weno5(q, s, scheme == 1);
}

}  // namespace erfk
