// Arithmetic-rate probes of the device (no counterpart in the paper): the
// measured ceilings against which the formal solution's roofline is reported.
// Each probe runs enough independent dependency chains per thread, and enough
// threads per SM, that the unit under test, not latency, bounds it:
//   0  FP32 fused multiply-add, scalar (fma.rn.f32)          flop/s (2 per FMA)
//   1  FP32 fused multiply-add, packed pairs (fma.rn.f32x2)  flop/s (4 per instruction)
//   2  special-function exponential (ex2.approx.ftz.f32)     results/s
//   3  special-function reciprocal (rcp.approx.ftz.f32)      results/s (each
//      followed by an add of 1, so that consecutive reciprocals cannot cancel;
//      the adds go to the FMA pipe, which has four times the issue rate)
//   4  FP64 fused multiply-add (fma.rn.f64)                  flop/s
// The values stay finite or saturate at inf; the rates do not depend on them.
#include <cuda_runtime.h>

#include <algorithm>

#include "rt_sc.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) probe_ffma(float *out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_ffma2(float *out, int iters, float a, float b) {
  unsigned long long x[kChains];
  float2 av = make_float2(a, a), bv = make_float2(b, b);
  const unsigned long long ab = *reinterpret_cast<unsigned long long *>(&av);
  const unsigned long long bb = *reinterpret_cast<unsigned long long *>(&bv);
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float2 v = make_float2(1e-3f * (threadIdx.x + c), 2e-3f * (threadIdx.x + c));
    x[c] = *reinterpret_cast<unsigned long long *>(&v);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(ab), "l"(bb));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float2 v = *reinterpret_cast<float2 *>(&x[c]);
    s += v.x + v.y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_ex2(float *out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_rcp(float *out, int iters) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("{\n\trcp.approx.ftz.f32 %0, %0;\n\tadd.ftz.f32 %0, %0, 0f3F800000;\n}" : "+f"(x[c]));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_dfma(float *out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// Best-of-three duration (ms) of one probe launch after a warm-up launch.
template <typename F>
cudaError_t time_best(F launch, float *ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  float best = 1e30f;
  launch();
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    best = std::min(best, t);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return e;
}

}  // namespace

extern "C" rt_status rt_measure_rates(double *rates, int n) {
  if (!rates || n < 1) return RT_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RT_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ERR_CUDA;
  // 8 blocks of 256 threads per SM: every SM holds 2048 threads of each probe
  const int blocks = sms * 8;
  const double threads = (double)blocks * kThreads;
  float *out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess) return RT_ERR_OOM;
  const double per_iter = (double)kChains * kUnroll;   // instructions per thread per iteration
  struct Probe {
    int iters;
    double ops_per_inst;
  };
  const Probe P[5] = {{4096, 2.0}, {4096, 4.0}, {1024, 1.0}, {1024, 1.0}, {128, 2.0}};
  rt_status st = RT_OK;
  for (int k = 0; k < std::min(n, 5) && st == RT_OK; ++k) {
    const int it = P[k].iters;
    float ms = 0.f;
    cudaError_t e;
    switch (k) {
      case 0: e = time_best([&] { probe_ffma<<<blocks, kThreads>>>(out, it, 0.9999f, 1e-7f); }, &ms); break;
      case 1: e = time_best([&] { probe_ffma2<<<blocks, kThreads>>>(out, it, 0.9999f, 1e-7f); }, &ms); break;
      case 2: e = time_best([&] { probe_ex2<<<blocks, kThreads>>>(out, it); }, &ms); break;
      case 3: e = time_best([&] { probe_rcp<<<blocks, kThreads>>>(out, it); }, &ms); break;
      default: e = time_best([&] { probe_dfma<<<blocks, kThreads>>>(out, it, 0.9999, 1e-7); }, &ms); break;
    }
    if (e != cudaSuccess || ms <= 0.f) {
      st = RT_ERR_CUDA;
      break;
    }
    rates[k] = threads * per_iter * it * P[k].ops_per_inst / (ms * 1e-3);
  }
  cudaFree(out);
  return st;
}
