// 1D march of Scheme 1 (Sec. 3.1.5) resident in one CTA.
//
// A 1D mesh of up to a few thousand nodes is far too small to fill the GPU,
// and one launch per step costs more than the step itself.  Here one CTA
// holds u (two buffers) and the scaled PCHIP slopes of Eq. (e300) in shared
// memory and runs every time step between two CTA barriers:
//   1. slopes of u^{n+1} (the end rule after Eq. (e300) gives node 0 the
//      slope of node 1 and node n-1 that of node n-2, the harmonic mean
//      being symmetric, so an end node uses its neighbour's differences);
//   2. per interior node the Gauss-Hermite points of Eq. (e31) (constant
//      drift: the shift is the same at every node), the exit value 1 outside
//      the closed interval (Eq. (e24)), the cubic Hermite value of
//      Eq. (Lag11), and the sum u_j + sum_q w_q (Itilde_q - u_j); the end
//      nodes hold 1 (Eq. (e3)).
// The input is read completely before the first barrier and the output
// written after the last, so u_in may alias u_out.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {

template <typename T, int Q>
__global__ void __launch_bounds__(1024) k_march1d(const Step1D<T> a, const T* u_in, T* u_out,
                                                  T* snaps, int stride, int steps) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = a.nx, tid = threadIdx.x, nt = blockDim.x;
  T* cur = reinterpret_cast<T*>(smem);
  T* nxt = cur + nx;
  T* D = nxt + nx;
  for (int i = tid; i < nx; i += nt)
    cur[i] = u_in ? u_in[i] : ((i == 0 || i == nx - 1) ? T(1) : T(0));
  __syncthreads();
  for (int m = 1; m <= steps; ++m) {
    for (int i = tid; i < nx; i += nt) {
      const int c = i + (i == 0) - (i == nx - 1);
      D[i] = pchip_scaled(cur[c] - cur[c - 1], cur[c + 1] - cur[c]);
    }
    __syncthreads();
    for (int i = tid; i < nx; i += nt) {
      if (i == 0 || i == nx - 1) {
        nxt[i] = T(1);
        continue;
      }
      const T uj = cur[i];
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T d = a.cdx + a.g[q];
        if (d < T(-i) || d > T(nx - 1 - i)) {
          acc += a.w[q] * (T(1) - uj);
          continue;
        }
        const T fl = floor(d);
        int c = i + (int)fl;
        T t = d - fl;
        if (c > nx - 2) {  // a point exactly on the upper end: t = 1 of the last cell
          c = nx - 2;
          t = T(1);
        }
        const T u0 = cur[c], u1 = cur[c + 1];
        const T t2 = t * t, omt = T(1) - t;
        const T v = (u0 - uj) + (t2 * (T(3) - T(2) * t)) * (u1 - u0) + (t * omt * omt) * D[c] -
                    (t2 * omt) * D[c + 1];
        acc += a.w[q] * v;
      }
      nxt[i] = uj + acc;
    }
    __syncthreads();
    if (snaps && stride > 0 && m % stride == 0) {
      T* s = snaps + (int64_t)(m / stride - 1) * nx;
      for (int i = tid; i < nx; i += nt) s[i] = nxt[i];
    }
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int i = tid; i < nx; i += nt) u_out[i] = cur[i];
}

template <typename T, int Q>
cudaError_t launch_q(const Step1D<T>& a, const T* u_in, T* u_out, T* snaps, int stride, int steps,
                     cudaStream_t s) {
  const int threads = a.nx >= 1024 ? 1024 : (a.nx + 31) / 32 * 32;
  k_march1d<T, Q><<<1, threads, fk_march1d_smem(a.nx, (int)sizeof(T)), s>>>(a, u_in, u_out, snaps,
                                                                            stride, steps);
  return cudaGetLastError();
}

template <typename T, int Q>
cudaError_t attr_q() {
  return cudaFuncSetAttribute(k_march1d<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

}  // namespace

size_t fk_march1d_smem(int nx, int elem) { return (size_t)3 * nx * elem; }

template <typename T>
cudaError_t fk_launch_march1d(const Step1D<T>& a, int q, const T* u_in, T* u_out, T* snaps,
                              int stride, int steps, cudaStream_t s) {
  switch (q) {
#define FK_CASE(QQ) \
  case QQ: return launch_q<T, QQ>(a, u_in, u_out, snaps, stride, steps, s);
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
    FK_CASE(9) FK_CASE(10) FK_CASE(11) FK_CASE(12) FK_CASE(13) FK_CASE(14) FK_CASE(15) FK_CASE(16)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fk_prepare_march1d(int q, int elem) {
  switch (q) {
#define FK_CASE(QQ) \
  case QQ: return elem == 4 ? attr_q<float, QQ>() : attr_q<double, QQ>();
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
    FK_CASE(9) FK_CASE(10) FK_CASE(11) FK_CASE(12) FK_CASE(13) FK_CASE(14) FK_CASE(15) FK_CASE(16)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t fk_launch_march1d<float>(const Step1D<float>&, int, const float*, float*,
                                              float*, int, int, cudaStream_t);
template cudaError_t fk_launch_march1d<double>(const Step1D<double>&, int, const double*, double*,
                                               double*, int, int, cudaStream_t);
