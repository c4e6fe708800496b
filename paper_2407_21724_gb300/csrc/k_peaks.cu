// Arithmetic peaks of the device the context runs on, measured: FP32 and
// FP64 fused multiply-add throughput of the CUDA cores (plain and packed
// two-wide FP32).  The roofline of the CUDA-core kernels (near product,
// aggregation, receive and translation in FP32; the plain FP64 product) is
// taken against these rather than against unit counts times the clock.
//
// Each thread runs NCH independent multiply-add chains for `iters` steps on
// values the compiler cannot fold (they come from the arguments), then writes
// one sum so that no chain is dead.  The grid is 8 CTAs of 256 threads per
// SM; one warm-up launch precedes the timed one (CUDA events on one stream).
#include <cuda_runtime.h>

#include "smr_internal.h"

namespace smr {
namespace {

constexpr int NCH = 16;

__global__ void __launch_bounds__(256) k_peak_f32(int iters, float b, float c, float* out) {
  float a[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int t = 0; t < iters; ++t) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32x2(int iters, float b, float c, float* out) {
  float2 a[NCH / 2];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int i = 0; i < NCH / 2; ++i) a[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
  for (int t = 0; t < iters; ++t) {
#pragma unroll
    for (int i = 0; i < NCH / 2; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NCH / 2; ++i) s += a[i].x + a[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f64(int iters, double b, double c, double* out) {
  double a[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int t = 0; t < iters; ++t) {
#pragma unroll
    for (int i = 0; i < NCH; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace smr

using namespace smr;

extern "C" int smr_measure_peak(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return SMR_E_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return SMR_E_CUDA;
  const int blocks = 8 * sms, threads = 256;
  const int iters = kind == 2 ? 2048 : 32768;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return SMR_E_OOM;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SMR_OK;
  float ms = 0.f;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = SMR_E_CUDA;
  } else {
    for (int rep = 0; rep < 2 && rc == SMR_OK; ++rep) {   // warm-up, then the timed launch
      cudaEventRecord(e0, st);
      if (kind == 0)
        k_peak_f32<<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-4f, (float*)out);
      else if (kind == 1)
        k_peak_f32x2<<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-4f, (float*)out);
      else
        k_peak_f64<<<blocks, threads, 0, st>>>(iters, 0.999, 1e-4, (double*)out);
      cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) rc = SMR_E_CUDA;
    }
    if (rc == SMR_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SMR_E_CUDA;
  }
  if (rc == SMR_OK) {
    const double flops = 2.0 * NCH * (double)iters * blocks * threads;
    *tflops = ms > 0 ? flops / (ms * 1e-3) / 1e12 : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}
