// Issue-rate probes for the arithmetic pipes the cell step runs on: FP32
// fused multiply-add, the multi-function unit (ex2, the base of every
// exponential of the FP32 cell models) and FP64 fused multiply-add. They
// give the ALU roofs against which the cell kernels are placed (the FP64
// plain step is bound by the FP64 pipe, not by HBM).
//
// Each thread runs kChains independent dependency chains so that the pipe,
// not the latency of one chain, bounds the loop; the grid fills every SM at
// full occupancy. The chains' results feed a comparison that is never true
// at run time, so the compiler keeps all of the work.
#include <cuda_runtime.h>

#include "kernels.h"

namespace ep {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) ffma_probe(float *sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = float(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) sink[0] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

// x <- 2^-x keeps every chain in [0.5, 1].
__global__ void __launch_bounds__(kProbeThreads) mufu_probe(float *sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = float(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = ex2_neg(x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) dfma_probe(double *sink, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = double(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) sink[0] = s;
}

}  // namespace

cudaError_t launch_alu_probe(int kind, int blocks, int iters, double *sink, cudaStream_t s, double *ops) {
    const double threads = double(blocks) * kProbeThreads * kChains * double(iters);
    switch (kind) {
    case 0:
        ffma_probe<<<blocks, kProbeThreads, 0, s>>>(reinterpret_cast<float *>(sink), iters, 0.999f, 0.001f);
        *ops = 2.0 * threads;   // one FMA = two flops
        break;
    case 1:
        mufu_probe<<<blocks, kProbeThreads, 0, s>>>(reinterpret_cast<float *>(sink), iters);
        *ops = threads;
        break;
    case 2:
        dfma_probe<<<blocks, kProbeThreads, 0, s>>>(sink, iters, 0.999, 0.001);
        *ops = 2.0 * threads;
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int alu_probe_threads() { return kProbeThreads; }

}  // namespace ep
