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
// The same update for a gate whose time constant is 1 / rate (rate = alpha +
// beta, or a multiple of it): no reciprocal of the rate is taken.
template <class R>
__device__ __forceinline__ R rush_larsen_rate(R y, R yinf, R rate, R dt) {
    return yinf + (y - yinf) * fexp(-dt * rate);
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

// Value of a parameter in the compute type: the FP64 copy for double, the
// FP32 copy for float.
template <class R> __device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// Error-free sum of two floats (Knuth's TwoSum), then renormalisation: adds
// the float d to the two-float value a = a.x + a.y, keeping ~48 significant
// bits. The sum uses only additions, so FMA contraction cannot alter it.
__device__ __forceinline__ float2 twofloat_add(float2 a, float d) {
    const float s = a.x + d;
    const float bp = s - a.x;
    const float err = (a.x - (s - bp)) + (d - bp);
    const float lo = a.y + err;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

// Slowly drifting concentrations ([Na]i, [K]i, SR calcium) live in 8-byte
// slots: an FP64 value in the plain path, a two-float compensated sum in the
// mixed path, so that FP32 increments accumulate without FP64 arithmetic.
// Rate a non-gating variable advances with over a step (V and the
// concentrations): forward Euler, f^n; or, with AB2 (second-order
// Adams-Bashforth, Sec. 4), 3/2 f^n - 1/2 f^{n-1} once the history exists.
// Slot k of the cell's history (h[k * st]) keeps f^n for the next step.
// Slots: 0 V, 1..5 the model's non-gating variables.
template <class R, bool AB2>
struct Rates {
    R *h = nullptr;        // NULL: this cell's job integrates by forward Euler
    long long st = 0;
    bool on = false;
    __device__ __forceinline__ R operator()(int k, R f) const {
        if constexpr (!AB2) {
            return f;
        } else {
            if (!h) return f;
            const R g = on ? R(1.5) * f - R(0.5) * h[k * st] : f;
            h[k * st] = f;
            return g;
        }
    }
};
// Where a cell model reads its state s^n and writes s^{n+1}: variable k at
// xi[k * si] / xo[k * so], 8-byte accumulator k at ai[k * si] / ao[k * so].
// In place (xi == xo) in global memory, or read from a shared-memory stage.
template <class R>
struct CellIO {
    const R *xi;
    const double *ai;
    long long si;
    R *xo;
    double *ao;
    long long so;
};

template <class R> struct Accum;
template <> struct Accum<double> {
    double v;
    __device__ __forceinline__ static Accum load(const double *p) { return Accum{*p}; }
    __device__ __forceinline__ double value() const { return v; }
    __device__ __forceinline__ void store_add(double *p, double d) const { *p = v + d; }
    __device__ __forceinline__ static void init(double *p, double x) { *p = x; }
    __device__ __forceinline__ static double read(const double *p) { return *p; }
};
template <> struct Accum<float> {
    float2 v;
    __device__ __forceinline__ static Accum load(const double *p) {
        return Accum{*reinterpret_cast<const float2 *>(p)};
    }
    __device__ __forceinline__ float value() const { return v.x; }
    __device__ __forceinline__ void store_add(double *p, float d) const {
        *reinterpret_cast<float2 *>(p) = twofloat_add(v, d);
    }
    __device__ __forceinline__ static void init(double *p, double x) {
        const float hi = float(x);
        *reinterpret_cast<float2 *>(p) = make_float2(hi, float(x - double(hi)));
    }
    __device__ __forceinline__ static double read(const double *p) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        return double(v.x) + double(v.y);
    }
};

}  // namespace ep
