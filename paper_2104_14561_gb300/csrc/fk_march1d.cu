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
//
// FP64 variant over a thread-block cluster: the same march split over up to
// 16 CTAs on separate SMs (GB300's FP64 rate makes one SM too slow).  CTA r
// owns a chunk of nodes and keeps u over the chunk plus a halo wide enough
// for the shifted points and their slope stencils; after each step every
// CTA stores its new values into its own buffer and into the halo copies of
// the CTAs whose windows hold them (distributed shared memory), and a
// cluster barrier ends the step.
#include <cooperative_groups.h>
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

// Cluster layout: CTA r owns nodes [r chunk, min((r+1) chunk, nx)) and
// holds global nodes [r chunk - halo, r chunk + chunk + halo) locally.
struct Cluster1D {
  int ctas, chunk, halo;
};

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_march1d_cluster(const Step1D<T> a, const Cluster1D cl,
                                                         const T* u_in, T* u_out, T* snaps,
                                                         int stride, int steps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = a.nx, tid = threadIdx.x, nt = blockDim.x;
  const int r = (int)cluster.block_rank();
  const int L = cl.chunk + 2 * cl.halo;  // local nodes
  const int g0 = r * cl.chunk - cl.halo;  // global node of local 0
  const int own0 = r * cl.chunk, own1 = min(own0 + cl.chunk, nx);
  T* const buf = reinterpret_cast<T*>(smem);  // two buffers of L nodes
  T* D = buf + 2 * L;
  T* terms = D + L;  // chunk x Q point terms
  for (int l = tid; l < L; l += nt) {
    const int g = g0 + l;
    const bool in = g >= 0 && g < nx;
    buf[l] = in ? (u_in ? u_in[g] : ((g == 0 || g == nx - 1) ? T(1) : T(0))) : T(0);
    buf[L + l] = T(0);
    D[l] = T(0);
  }
  cluster.sync();  // every CTA's buffers exist before any remote store
  int cur = 0;
  for (int m = 1; m <= steps; ++m) {
    const T* u = buf + cur * L;
    // slopes of the local nodes whose stencil is local (end rule: an end
    // node takes its neighbour's differences)
    for (int l = tid; l < L; l += nt) {
      const int g = g0 + l;
      if (g < 0 || g >= nx) continue;
      const int c = l + (g == 0) - (g == nx - 1);
      if (c < 1 || c > L - 2) continue;
      D[l] = pchip_scaled(u[c] - u[c - 1], u[c + 1] - u[c]);
    }
    __syncthreads();
    // one thread per (owned node, point): w_q (Itilde_q - u_j), or w_q (1 - u_j) on exit
    for (int e = tid; e < cl.chunk * Q; e += nt) {
      const int k = e / Q, q = e - k * Q;
      const int i = own0 + k;
      T term = T(0);
      if (i >= 1 && i <= nx - 2) {
        const int li = i - g0;
        const T uj = u[li];
        const T d = a.cdx + a.g[q];
        if (d < T(-i) || d > T(nx - 1 - i)) {
          term = a.w[q] * (T(1) - uj);
        } else {
          const T fl = floor(d);
          int c = i + (int)fl;
          T t = d - fl;
          if (c > nx - 2) {
            c = nx - 2;
            t = T(1);
          }
          const int lc = c - g0;
          const T u0 = u[lc], u1 = u[lc + 1];
          const T t2 = t * t, omt = T(1) - t;
          term = a.w[q] * ((u0 - uj) + (t2 * (T(3) - T(2) * t)) * (u1 - u0) +
                           (t * omt * omt) * D[lc] - (t2 * omt) * D[lc + 1]);
        }
      }
      terms[e] = term;
    }
    __syncthreads();
    // new values of the owned nodes, into this CTA's next buffer and into
    // the halo copies of the CTAs whose windows hold them
    T* nxt = buf + (cur ^ 1) * L;
    for (int k = tid; k < own1 - own0; k += nt) {
      const int i = own0 + k;
      T un;
      if (i == 0 || i == nx - 1) {
        un = T(1);
      } else {
        un = u[i - g0];
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) acc += terms[k * Q + q];
        un += acc;
      }
      nxt[i - g0] = un;
      for (int s2 = 0; s2 < cl.ctas; ++s2) {
        if (s2 == r) continue;
        const int l2 = i - (s2 * cl.chunk - cl.halo);
        if (l2 >= 0 && l2 < L) cluster.map_shared_rank(nxt, s2)[l2] = un;
      }
      if (snaps && stride > 0 && m % stride == 0) snaps[(int64_t)(m / stride - 1) * nx + i] = un;
    }
    cluster.sync();  // the step's stores are visible cluster-wide
    cur ^= 1;
  }
  for (int i = own0 + tid; i < own1; i += nt) u_out[i] = buf[cur * L + i - g0];
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

namespace {

template <typename T, int Q>
cudaError_t launch_cluster_q(const Step1D<T>& a, int ctas, const T* u_in, T* u_out, T* snaps,
                             int stride, int steps, cudaStream_t s) {
  Cluster1D cl;
  cl.ctas = ctas;
  cl.chunk = (a.nx + ctas - 1) / ctas;
  cl.halo = a.hx + 2;
  const int L = cl.chunk + 2 * cl.halo;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)(3 * L + cl.chunk * Q) * sizeof(T);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_march1d_cluster<T, Q>, a, cl, u_in, u_out, snaps, stride,
                            steps);
}

template <typename T, int Q>
cudaError_t attr_cluster_q() {
  cudaError_t e = cudaFuncSetAttribute(k_march1d_cluster<T, Q>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_march1d_cluster<T, Q>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// largest cluster this device runs for the kernel, at most 16
template <typename T, int Q>
int max_cluster_q() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 48 * 1024;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&n, k_march1d_cluster<T, Q>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n > 16 ? 16 : n;
}

}  // namespace

template <typename T>
cudaError_t fk_launch_march1d_cluster(const Step1D<T>& a, int q, int ctas, const T* u_in,
                                      T* u_out, T* snaps, int stride, int steps, cudaStream_t s) {
  switch (q) {
#define FK_CASE(QQ) \
  case QQ: return launch_cluster_q<T, QQ>(a, ctas, u_in, u_out, snaps, stride, steps, s);
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
    FK_CASE(9) FK_CASE(10) FK_CASE(11) FK_CASE(12) FK_CASE(13) FK_CASE(14) FK_CASE(15) FK_CASE(16)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

// Opts the cluster kernel into 16-CTA clusters and returns the largest
// cluster the device runs for it (0: none).
int fk_prepare_march1d_cluster(int q, int elem) {
  switch (q) {
#define FK_CASE(QQ)                                                              \
  case QQ:                                                                       \
    if (elem == 4) {                                                             \
      if (attr_cluster_q<float, QQ>() != cudaSuccess) return cudaGetLastError(), 0; \
      return max_cluster_q<float, QQ>();                                         \
    } else {                                                                     \
      if (attr_cluster_q<double, QQ>() != cudaSuccess) return cudaGetLastError(), 0; \
      return max_cluster_q<double, QQ>();                                        \
    }
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
    FK_CASE(9) FK_CASE(10) FK_CASE(11) FK_CASE(12) FK_CASE(13) FK_CASE(14) FK_CASE(15) FK_CASE(16)
#undef FK_CASE
    default: return 0;
  }
}

template cudaError_t fk_launch_march1d_cluster<float>(const Step1D<float>&, int, int, const float*,
                                                      float*, float*, int, int, cudaStream_t);
template cudaError_t fk_launch_march1d_cluster<double>(const Step1D<double>&, int, int,
                                                       const double*, double*, double*, int, int,
                                                       cudaStream_t);

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
