// fk_measure_fma_rate: the fused multiply-add throughput of the current
// device, for the rooflines of the ALU-bound march kernels (a measurement
// aid with no counterpart in the paper).
//
// Every SM runs resident CTAs whose threads each advance eight independent
// FMA chains from registers (no memory traffic inside the loop), so the
// issue of the FMA pipe is the only limit.  The FP32 rate is measured twice:
// with scalar FFMA and with the packed f32x2 form (__ffma2_rn), which does
// two FMAs per instruction; the step kernels use both.  The kernel time
// comes from CUDA events on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fk_internal.h"

namespace {

__device__ double g_fma_sink;  // keeps the chains' results observable

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T x, T y) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = fma(a[c], x, y);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == (T)-1.2345e30) g_fma_sink = (double)s;  // never true; not removable
}

__global__ void __launch_bounds__(256) k_fma2_chains(int iters, float x, float y) {
  float2 a[8];
  const float2 xx = make_float2(x, x), yy = make_float2(y, y);
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = make_float2((threadIdx.x + c) * 1e-3f, c * 1e-3f);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = __ffma2_rn(a[c], xx, yy);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c].x + a[c].y;
  if (s == -1.2345e30f) g_fma_sink = (double)s;
}

cudaError_t launch(int kind, int blocks, int iters, cudaStream_t s) {
  const float xf = 0.999999f, yf = 1e-7f;
  if (kind == 0) k_fma_chains<float><<<blocks, 256, 0, s>>>(iters, xf, yf);
  else if (kind == 1) k_fma2_chains<<<blocks, 256, 0, s>>>(iters, xf, yf);
  else k_fma_chains<double><<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace

extern "C" fk_status fk_measure_fma_rate(fk_precision prec, int packed, double seconds,
                                         double* flop_per_s, cudaStream_t stream) {
  if (!flop_per_s || (prec != FK_FP32 && prec != FK_FP64) || (packed && prec != FK_FP32) ||
      !(seconds > 0.0) || seconds > 10.0)
    return FK_ERR_INVALID_ARG;
  *flop_per_s = 0.0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
    return FK_ERR_CUDA;
  const int kind = prec == FK_FP64 ? 2 : (packed ? 1 : 0);
  const int blocks = sms * (per_sm / 256);  // every thread slot of every SM
  // flop of one loop iteration of one thread: 16 x 8 FMAs (x2 lanes packed)
  const double flop_iter = 2.0 * 16 * 8 * (kind == 1 ? 2 : 1);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FK_ERR_CUDA;
  }
  fk_status st = FK_OK;
  int iters = kind == 2 ? 4 : 64;
  double rate = 0.0;
  for (int attempt = 0; attempt < 8 && st == FK_OK; ++attempt) {
    if (launch(kind, blocks, iters, stream) != cudaSuccess) {  // warm-up / clocks up
      st = FK_ERR_CUDA;
      break;
    }
    cudaEventRecord(e0, stream);
    if (launch(kind, blocks, iters, stream) != cudaSuccess) {
      st = FK_ERR_CUDA;
      break;
    }
    cudaEventRecord(e1, stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = FK_ERR_CUDA;
      break;
    }
    rate = flop_iter * iters * blocks * 256.0 / (ms * 1e-3);
    if (ms * 1e-3 >= 0.5 * seconds) break;
    // scale the loop towards the requested duration (bounded growth)
    const double grow = ms > 0.f ? seconds / (ms * 1e-3) : 64.0;
    const double next = iters * (grow < 64.0 ? grow : 64.0);
    if (next > 2.0e9) break;
    iters = (int)next + 1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == FK_OK) *flop_per_s = rate;
  return st;
}
