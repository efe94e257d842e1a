// Arithmetic helpers shared by the device cell models, overloaded on the
// compute type (float for EP_FP32_MIXED, double for EP_FP64_PLAIN).
#pragma once
#include <cuda_runtime.h>

namespace ep {

__device__ __forceinline__ float fexp(float x) { return expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float flog(float x) { return logf(x); }
__device__ __forceinline__ double flog(double x) { return log(x); }
__device__ __forceinline__ float fsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double fexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float fpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double fpow(double x, double y) { return pow(x, y); }

// Rush-Larsen update: exact solution of dy/dt = (yinf - y)/tau over dt with
// yinf and tau frozen at V^n (Sec. 3.2).
template <class R>
__device__ __forceinline__ R rush_larsen(R y, R yinf, R tau, R dt) {
    return yinf + (y - yinf) * fexp(-dt / tau);
}

// Logistic 1/(1 + exp(x)).
template <class R>
__device__ __forceinline__ R logistic(R x) {
    return R(1) / (R(1) + fexp(x));
}

// x / expm1(x), continuous at 0 where it is 1.
template <class R>
__device__ __forceinline__ R x_over_expm1(R x) {
    return x == R(0) ? R(1) : x / fexpm1(x);
}

// Forward-Euler step of a rapidly buffered compartment, in increment form.
// The buffered total T(c) = c + B c/(c + K) advances by dtot; the free
// concentration moves by the delta with T(c + delta) = T(c) + dtot, the
// root continuous at dtot = 0 of
//     u delta^2 + (u^2 + B K - dtot u) delta - dtot u^2 = 0,   u = c + K.
// Computing the increment (not the new total) keeps the FP32 rounding
// relative to the change rather than to the concentration.
template <class R>
__device__ __forceinline__ R buffered_increment(R c, R dtot, R B, R K) {
    const R u = c + K;
    const R p = u * u + B * K - dtot * u;
    const R disc = fsqrt(p * p + R(4) * u * u * u * dtot);
    return p > R(0) ? R(2) * dtot * u * u / (p + disc) : (disc - p) / (R(2) * u);
}

}  // namespace ep
