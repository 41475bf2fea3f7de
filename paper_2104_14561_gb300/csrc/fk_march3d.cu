// Step of Scheme 1 (Sec. 3.1.5) on a 3D tensor mesh, for sm_103a.
//
// The tensor extension of Sec. 3.1.3 to d = 3.  Drift and sigma are taken
// at the node (Eq. (e31)) and sigma is diagonal, so the Q^3 Gauss-Hermite
// points of node j form a grid X_p x Y_q x Z_r.  The zero-twist tricubic
// Hermite interpolant of Eq. (Lag11) holds, per corner node, the value and
// the three first partials (no cross derivatives), each times a product of
// 1D Hermite functions, so the quadrature sum splits into 1D weights over a
// W x W x W window of nodes:
//
//   sum_{p,q,r} w_p w_q w_r Itilde(X_p, Y_q, Z_r)
//     = sum_{a,b,c} u V^x_a V^y_b V^z_c + hx u_x D^x_a V^y_b V^z_c
//                 + hy u_y V^x_a D^y_b V^z_c + hz u_z V^x_a V^y_b D^z_c,
//
// V^x_a = sum_p w_p (value basis of node a at X_p), D^x_a the same with the
// slope basis (and along y, z).  A point exits (Eq. (e24)) when any of its
// coordinates leaves the closed box.  The inside points are then a product
// of per-axis sets, so dropping each axis's exiting coordinates from its 1D
// weights keeps the sum separable; the exit mass is 1 - prod_m (1 - E_m),
// E_m the weight of axis m's dropped coordinates.  As in 2D the window part
// is written in the increment form u_j + sum w (Itilde - u_j).
//
// Two launches per step:
//  * k_rec3d writes one record {u, hx u_x, hy u_y, hz u_z} per node (the
//    scaled PCHIP slopes of Eq. (e300) with the end rule that gives node 0
//    the slope of node 1 and node n-1 that of node n-2), and 1 into u^n at
//    every boundary node (Eq. (e3));
//  * k_step3d forms each interior node's 1D weights in registers and sums
//    the W^3 records of its window, read through L1/L2 (a warp's 32
//    consecutive x-nodes read overlapping, contiguous windows).
// Positions are taken relative to the node in cells: point p of axis m is
// at i_m + rel_p with rel_p = b_m dt / h_m + sigma_m sqrt(2 dt) a_p / h_m.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {

constexpr int kRecThreads = 128;

template <typename T>
__device__ __forceinline__ T floor_t(T x);
template <>
__device__ __forceinline__ float floor_t<float>(float x) { return floorf(x); }
template <>
__device__ __forceinline__ double floor_t<double>(double x) { return floor(x); }

// Records and boundary values of one field.
template <typename T>
__global__ void __launch_bounds__(kRecThreads) k_rec3d(const Step3D<T> a) {
  const int i = blockIdx.x * kRecThreads + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= a.nx) return;
  const int64_t sy = a.nx, sz = (int64_t)a.nx * a.ny;
  const int64_t node = (int64_t)k * sz + (int64_t)j * sy + i;
  const T* u = a.u_in;
  // slope of Eq. (e300) along one axis at index idx (n nodes, stride st)
  auto slope = [&](int idx, int n, int64_t st) {
    const int c = idx < 1 ? 1 : (idx > n - 2 ? n - 2 : idx);
    const T* b = u + node + (int64_t)(c - idx) * st;
    const T um = b[-st], u0 = b[0], up = b[st];
    return pchip_fast(u0 - um, up - u0);
  };
  V4<T> r;
  r.x = u[node];
  r.y = slope(i, a.nx, 1);
  r.z = slope(j, a.ny, sy);
  r.w = slope(k, a.nz, sz);
  a.rec[node] = r;
  if (i == 0 || i == a.nx - 1 || j == 0 || j == a.ny - 1 || k == 0 || k == a.nz - 1) {
    a.u_out[node] = T(1);
    if (a.snap) a.snap[node] = T(1);
  }
}

// The 1D weights of one axis over its window [org, org + W): node i of n,
// points at i + sh + gs a_q.  Returns the exit weight E; sets bad when an
// inside point's cell falls outside the window (cannot happen for the W the
// plan chooses; the check keeps every read in bounds regardless).
template <typename T, int W>
__device__ __forceinline__ T axis_weights(const Step3D<T>& a, int i, int n, T sh, T gs,
                                          T (&V)[W], T (&D)[W], int& org, unsigned& bad) {
#pragma unroll
  for (int t = 0; t < W; ++t) {
    V[t] = T(0);
    D[t] = T(0);
  }
  T E = T(0);
  const T lo = T(-i), hi = T(n - 1 - i);  // the box, relative to the node
  // the abscissae ascend and gs >= 0: point 0 is the leftmost
  int o = i + (int)floor_t(sh + gs * a.ga[0]);
  o = o < 0 ? 0 : o;
  o = o > n - W ? n - W : o;
  org = o;
#pragma unroll
  for (int q = 0; q < FK_MAXQ_2D; ++q) {
    if (q < a.q) {
      const T rel = sh + gs * a.ga[q];
      const T wq = a.gw[q];
      const bool in = !(rel < lo || rel > hi);
      const T fl = floor_t(rel);
      int c = i + (int)fl;
      T s = rel - fl;
      if (c == n - 1) {  // on the upper face: the last cell at s = 1
        c -= 1;
        s = T(1);
      }
      const int off = c - o;
      const bool ok = off >= 0 && off <= W - 2;
      if (in && !ok) bad = 1u;
      E += in ? T(0) : wq;
      const T wi = (in && ok) ? wq : T(0);
      // cubic Hermite basis on a unit cell (Sec. 3.1.3)
      const T s2 = s * s, r1 = T(1) - s;
      const T h00 = (T(1) + T(2) * s) * r1 * r1, h01 = s2 * (T(3) - T(2) * s);
      const T h10 = s * r1 * r1, h11 = -s2 * r1;
#pragma unroll
      for (int t = 0; t < W; ++t) {
        V[t] += (t == off) ? wi * h00 : ((t == off + 1) ? wi * h01 : T(0));
        D[t] += (t == off) ? wi * h10 : ((t == off + 1) ? wi * h11 : T(0));
      }
    }
  }
  return E;
}

template <typename T, int W>
__global__ void __launch_bounds__(kRecThreads) k_step3d(const Step3D<T> a) {
  const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 1 + blockIdx.y, k = 1 + blockIdx.z;
  if (i > a.nx - 2) return;
  const int64_t sy = a.nx, sz = (int64_t)a.nx * a.ny;
  const int64_t node = (int64_t)k * sz + (int64_t)j * sy + i;

  // 1D weights per axis (constant drift: shift and scale are plan constants)
  T Vx[W], Dx[W], Vy[W], Dy[W], Vz[W], Dz[W];
  int ox, oy, oz;
  unsigned bad = 0;
  const T Ex = axis_weights<T, W>(a, i, a.nx, a.cd[0], a.gs[0], Vx, Dx, ox, bad);
  const T Ey = axis_weights<T, W>(a, j, a.ny, a.cd[1], a.gs[1], Vy, Dy, oy, bad);
  const T Ez = axis_weights<T, W>(a, k, a.nz, a.cd[2], a.gs[2], Vz, Dz, oz, bad);

  const V4<T>* R = a.rec;
  const T uj = R[node].x;
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const T vz = Vz[c], dz = Dz[c];
    const V4<T>* plane = R + (int64_t)(oz + c) * sz + (int64_t)oy * sy + ox;
    T P = T(0), Pz = T(0);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const V4<T>* row = plane + (int64_t)b * sy;
      T s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const V4<T> r = row[t];
        s1 += Vx[t] * (r.x - uj) + Dx[t] * r.y;
        s2 += Vx[t] * r.z;
        s3 += Vx[t] * r.w;
      }
      P += Vy[b] * s1 + Dy[b] * s2;
      Pz += Vy[b] * s3;
    }
    acc += vz * P + dz * Pz;
  }
  // exit mass 1 - (1 - Ex)(1 - Ey)(1 - Ez), exactly 0 when no point exits
  const T ex = Ex + (T(1) - Ex) * (Ey + (T(1) - Ey) * Ez);
  const T un = uj + acc + (T(1) - uj) * ex;
  a.u_out[node] = un;
  if (a.snap) a.snap[node] = un;
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

template <typename T, int W>
cudaError_t launch_w(const Step3D<T>& a, cudaStream_t s) {
  const int in = a.nx - 2;
  const int bx = in <= 32 ? 32 : (in <= 64 ? 64 : kRecThreads);
  const dim3 grid((unsigned)((in + bx - 1) / bx), (unsigned)(a.ny - 2), (unsigned)(a.nz - 2));
  k_step3d<T, W><<<grid, bx, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t fk_launch_step3d(const Step3D<T>& a, cudaStream_t s) {
  {
    const dim3 grid((unsigned)((a.nx + kRecThreads - 1) / kRecThreads), (unsigned)a.ny,
                    (unsigned)a.nz);
    k_rec3d<T><<<grid, kRecThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  switch (a.w3) {
    case 3: return launch_w<T, 3>(a, s);
    case 4: return launch_w<T, 4>(a, s);
    case 5: return launch_w<T, 5>(a, s);
    case 6: return launch_w<T, 6>(a, s);
    case 7: return launch_w<T, 7>(a, s);
    case 8: return launch_w<T, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t fk_launch_step3d<float>(const Step3D<float>&, cudaStream_t);
template cudaError_t fk_launch_step3d<double>(const Step3D<double>&, cudaStream_t);
