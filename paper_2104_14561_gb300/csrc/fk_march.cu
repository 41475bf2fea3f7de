// Matrix-free fused step of Scheme 1 (Sec. 3.1.5) for sm_103a.
//
// One launch computes u^n from u^{n+1} on the whole mesh.  Each CTA owns a
// tile of interior output nodes and does, for that tile:
//   1. stage u^{n+1} over the tile plus a halo wide enough for every shifted
//      point of Eq. (e31) into shared memory (coalesced loads; the field of
//      a 1025x513 mesh is L2-resident between steps);
//   2. compute the PCHIP nodal slopes of Eq. (e300) (the map F^n of
//      Eq. (e34)) for the staged nodes and pack, per cell and row, the
//      record {u_c, u_{c+1}-u_c, h u'_c, h u'_{c+1}} and {h u_y,c,
//      h u_y,c+1 - h u_y,c} that one Hermite evaluation reads;
//   3. per output node: the drift (Eq. (ref-X)) from per-row/per-column
//      tables, the tensor Gauss-Hermite shifted points of Eq. (e31) in cell
//      units, the exit test (value 1 outside the closed box, Eq. (e24)),
//      the zero-twist bicubic Hermite value of Eq. (Lag11) from 4 vector
//      shared-memory loads, and the quadrature sum of Eq. (e304);
//   4. store u^n, and 1 on the adjacent boundary nodes (Eq. (e3)).
//
// Precision: the sum is formed as u_j + sum_q w_q (Itilde_q - u_j), which is
// the same number in exact arithmetic (the weights sum to 1 and the
// Hermite value functions form a partition of unity) but keeps the rounding
// error proportional to the per-step change instead of to u itself; without
// it an FP32 march of 2000 steps drifts by ~1e-4 near u = 1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_internal.h"

namespace {

// Scaled PCHIP slope h*u'_j from the two neighbouring differences
// (Eq. (e300)): 0 unless both have the same strict sign, else their
// harmonic mean 2 dl dr / (dl + dr).
template <typename T>
__device__ __forceinline__ T pchip_scaled(T dl, T dr) {
  const T p = dl * dr;
  return p > T(0) ? (T(2) * p) / (dl + dr) : T(0);
}

// Scaled slope along a staged line at local position l of a node whose
// global index on that axis is g (0..n-1); stride is the distance between
// neighbours in the staged array.  End nodes use the end rule stated after
// Eq. (e300): node 0 takes (delta_0, delta_1), node n-1 takes
// (delta_{n-2}, delta_{n-3}).  Nodes outside the mesh get 0 (never read).
template <typename T>
__device__ __forceinline__ T slope_line(const T* u, int l, int stride, int g, int n) {
  if (g < 0 || g >= n) return T(0);
  const T* c = u + l * stride;
  if (g == 0) return pchip_scaled(c[stride] - c[0], c[2 * stride] - c[stride]);
  if (g == n - 1) return pchip_scaled(c[0] - c[-stride], c[-stride] - c[-2 * stride]);
  return pchip_scaled(c[0] - c[-stride], c[stride] - c[0]);
}

// Cell and fractional position of a shifted point along one axis, in index
// space: node index k plus shift d.  Returns true when the point is outside
// the closed interval [0, n-1] (exit).  The cell is clamped to n-2 so that a
// point exactly on the upper face uses t = 1 of the last cell.
template <typename T>
__device__ __forceinline__ bool locate(int k, T d, int n, int* cell, T* t) {
  const bool out = (d < T(-k)) || (d > T(n - 1 - k));
  const T fl = floor(d);
  int c = k + (int)fl;
  T tt = d - fl;
  if (c > n - 2) {
    c = n - 2;
    tt = T(1);
  }
  *cell = c;
  *t = tt;
  return out;
}

// Slope of Eq. (e300) from two neighbouring differences, in the FP32 path
// with a fast reciprocal (the slope feeds an O(h) correction term, so a
// 2-ulp quotient is far inside the 1e-5 parity budget); FP64 divides exactly.
template <typename T>
__device__ __forceinline__ T pchip_fast(T dl, T dr) { return pchip_scaled(dl, dr); }
template <>
__device__ __forceinline__ float pchip_fast<float>(float dl, float dr) {
  const float p = dl * dr;
  return p > 0.f ? __fdividef(2.f * p, dl + dr) : 0.f;
}
template <typename T>
__device__ __forceinline__ T slope_fast(const T* u, int l, int stride, int g, int n) {
  if (g < 0 || g >= n) return T(0);
  const T* c = u + l * stride;
  if (g == 0) return pchip_fast(c[stride] - c[0], c[2 * stride] - c[stride]);
  if (g == n - 1) return pchip_fast(c[0] - c[-stride], c[-stride] - c[-2 * stride]);
  return pchip_fast(c[0] - c[-stride], c[stride] - c[0]);
}

// MINB = CTAs of 256 threads per SM that the register budget is sized for
// (4 -> <= 64 registers, 3 -> <= 85, 2 -> <= 128); the plan's autotuner
// picks the variant together with the tile height.

// Tiles are 32 nodes wide (one warp per tile row) and a multiple of 8 rows
// high (ty = 8 * passes); every staging loop walks rows by warp and columns
// by lane, so no index needs an integer division.
template <typename T, int Q, int MINB>
__global__ void __launch_bounds__(FK_THREADS, MINB) k_step2d(const Step2D<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  V2<T>* S = reinterpret_cast<V2<T>*>(R + lx * lyr);
  T* U = reinterpret_cast<T*>(S + lx * lyr);
  T* DX = U + lx * ly;
  T* DY = DX + lx * ly;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int i0 = 1 + blockIdx.x * 32;  // first interior output node of the tile
  const int k0 = 1 + blockIdx.y * a.ty;
  const int gi0 = i0 - a.hx - 1;  // global node of staged column 0
  const int gk0 = k0 - a.hy - 1;

  // 1. stage u^{n+1} (zero outside the mesh; never read there)
  for (int lk = warp; lk < ly; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const bool rowin = gk >= 0 && gk < a.ny;
    const T* src = a.u_in + (int64_t)gk * a.nx;
    for (int li = lane; li < lx; li += 32) {
      const int gi = gi0 + li;
      U[lk * lx + li] = (rowin && gi >= 0 && gi < a.nx) ? src[gi] : T(0);
    }
  }
  __syncthreads();

  // 2. scaled PCHIP slopes h u_x, h u_y of the staged nodes 1..lx-2, 1..ly-2
  for (int lk = 1 + warp; lk <= ly - 2; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const T* row = U + lk * lx;
    for (int li = 1 + lane; li <= lx - 2; li += 32) {
      DX[lk * lx + li] = slope_fast(row, li, 1, gi0 + li, a.nx);
      DY[lk * lx + li] = slope_fast(U + li, lk, lx, gk, a.ny);
    }
  }
  __syncthreads();

  // 3. packed cell records (column-major, odd pitch: conflict-free)
  for (int lk = 1 + warp; lk <= ly - 2; lk += FK_THREADS / 32) {
    for (int lc = 1 + lane; lc <= lx - 3; lc += 32) {
      const int o = lk * lx + lc;
      const T u0 = U[o], u1 = U[o + 1];
      V4<T> r;
      r.x = u0; r.y = u1 - u0; r.z = DX[o]; r.w = DX[o + 1];
      V2<T> s;
      s.x = DY[o]; s.y = DY[o + 1] - DY[o];
      R[lc * lyr + lk] = r;
      S[lc * lyr + lk] = s;
    }
  }
  __syncthreads();

  // 4. one output node per thread and pass: column i0 + lane, row k0 + warp + 8 m
  const int i = i0 + lane;
  const int li = i - gi0;
  const bool colok = i <= a.nx - 2;
  T cx0 = T(0), cx1 = T(0), cx2 = T(0), cx3 = T(0);
  if (a.family == FK_CELLULAR_FLOW && colok) {
    const T* ct = a.col_tab + 4 * (int64_t)i;
    cx0 = ct[0]; cx1 = ct[1]; cx2 = ct[2]; cx3 = ct[3];
  }
  const T nlo_x = T(-i), nhi_x = T(a.nx - 1 - i);
  unsigned bad = 0;
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (!colok || k > a.ny - 2) continue;
    const int lk = k - gk0;
    const T uj = R[li * lyr + lk].x;
    T dx, dy;
    if (a.family == FK_CELLULAR_FLOW) {
      const T* rt = a.row_tab + 2 * (int64_t)k;
      dx = a.kx * rt[0] * (a.A * cx0 + a.e1 * cx1);
      dy = a.ky * rt[1] * (a.A * cx2 + a.e2 * cx3);
    } else {
      dx = a.cdx;
      dy = a.cdy;
    }
    // y factors of every query row, weights folded in
    const T nlo_y = T(-k), nhi_y = T(a.ny - 1 - k);
    int rq[Q];
    T w0[Q], w1[Q], w2[Q], w3[Q];
    T exit_y = T(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T d = dy + a.gy[q];
      const bool out = (d < nlo_y) || (d > nhi_y);
      const T fl = floor(d);
      int c = k + (int)fl;
      T t = d - fl;
      if (c > a.ny - 2) {
        c = a.ny - 2;
        t = T(1);
      }
      int lc = c - gk0;
      if ((unsigned)(lc - 1) > (unsigned)(ly - 4)) {
        bad |= out ? 0u : 1u;
        lc = lk;
      }
      const T wq = out ? T(0) : a.w[q];
      exit_y += a.w[q] - wq;
      rq[q] = out ? lk : lc;
      const T t2 = t * t, omt = T(1) - t;
      w0[q] = wq;
      w1[q] = wq * (t2 * (T(3) - T(2) * t));  // h01
      w2[q] = wq * (t * omt * omt);            // h10
      w3[q] = -wq * (t2 * omt);                // h11
    }
    const T om = T(1) - uj;
    T acc = T(0);
#pragma unroll 1
    for (int p = 0; p < Q; ++p) {
      const T d = dx + a.gx[p];
      if ((d < nlo_x) || (d > nhi_x)) {
        acc += a.w[p] * om;
        continue;
      }
      const T fl = floor(d);
      int c = i + (int)fl;
      T t = d - fl;
      if (c > a.nx - 2) {
        c = a.nx - 2;
        t = T(1);
      }
      int lc = c - gi0;
      if ((unsigned)(lc - 1) > (unsigned)(lx - 4)) {
        bad |= 1u;
        lc = li;
      }
      const T t2 = t * t, omt = T(1) - t;
      const T h01 = t2 * (T(3) - T(2) * t), h10 = t * omt * omt, h11 = -(t2 * omt);
      const V4<T>* Rc = R + lc * lyr;
      const V2<T>* Sc = S + lc * lyr;
      T accp = exit_y * om;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const V4<T> r0 = Rc[rq[q]];
        const V4<T> r1 = Rc[rq[q] + 1];
        const V2<T> s0 = Sc[rq[q]];
        const V2<T> s1 = Sc[rq[q] + 1];
        const T a0 = (r0.x - uj) + h01 * r0.y + h10 * r0.z + h11 * r0.w;
        const T a1 = (r1.x - uj) + h01 * r1.y + h10 * r1.z + h11 * r1.w;
        const T b0 = s0.x + h01 * s0.y;
        const T b1 = s1.x + h01 * s1.y;
        accp += w0[q] * a0;
        accp += w1[q] * (a1 - a0);
        accp += w2[q] * b0;
        accp += w3[q] * b1;
      }
      acc += a.w[p] * accp;
    }
    const T un = uj + acc;
    const int64_t nx = a.nx;
    a.u_out[(int64_t)k * nx + i] = un;
    if (a.snap) a.snap[(int64_t)k * nx + i] = un;
    // 5. boundary nodes adjacent to this interior node hold 1 (Eq. (e3))
    const bool L = (i == 1), Rt = (i == a.nx - 2), B = (k == 1), Tp = (k == a.ny - 2);
    if (L | Rt | B | Tp) {
      // On a mesh with 3 nodes along an axis the single interior line is
      // next to both faces of that axis, so every flag is tested on its own.
      const int64_t top = (int64_t)(a.ny - 1) * nx, row = (int64_t)k * nx;
      auto one = [&](int64_t j) {
        a.u_out[j] = T(1);
        if (a.snap) a.snap[j] = T(1);
      };
      if (L) one(row);
      if (Rt) one(row + nx - 1);
      if (B) one(i);
      if (Tp) one(top + i);
      if (L & B) one(0);
      if (Rt & B) one(nx - 1);
      if (L & Tp) one(top);
      if (Rt & Tp) one(top + nx - 1);
    }
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// 1D step: same structure with a record {u_c, u_{c+1}-u_c, h u'_c, h u'_{c+1}}
// per staged cell.
template <typename T, int Q>
__global__ void __launch_bounds__(FK_THREADS) k_step1d(const Step1D<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  T* U = reinterpret_cast<T*>(R + lx);
  const int i0 = 1 + blockIdx.x * a.tx;
  const int gi0 = i0 - a.hx - 1;
  for (int e = threadIdx.x; e < lx; e += blockDim.x) {
    const int gi = gi0 + e;
    U[e] = (gi >= 0 && gi < a.nx) ? a.u_in[gi] : T(0);
  }
  __syncthreads();
  for (int lc = 1 + threadIdx.x; lc <= lx - 3; lc += blockDim.x) {
    const int gi = gi0 + lc;
    V4<T> r;
    r.x = U[lc];
    r.y = U[lc + 1] - U[lc];
    r.z = slope_line(U, lc, 1, gi, a.nx);
    r.w = slope_line(U, lc + 1, 1, gi + 1, a.nx);
    R[lc] = r;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < a.tx; e += blockDim.x) {
    const int i = i0 + e;
    if (i > a.nx - 2) continue;
    const int li = i - gi0;
    const T uj = R[li].x;
    const T om = T(1) - uj;
    T acc = T(0);
    unsigned bad = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int c;
      T t;
      const bool out = locate(i, a.cdx + a.g[q], a.nx, &c, &t);
      if (out) {
        acc += a.w[q] * om;
        continue;
      }
      int lc = c - gi0;
      if (lc < 1 || lc > lx - 3) {
        bad |= 1u;
        lc = li;
      }
      const T t2 = t * t, omt = T(1) - t;
      const V4<T> r = R[lc];
      const T v = (r.x - uj) + (t2 * (T(3) - T(2) * t)) * r.y + (t * omt * omt) * r.z - (t2 * omt) * r.w;
      acc += a.w[q] * v;
    }
    if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
    const T un = uj + acc;
    a.u_out[i] = un;
    if (a.snap) a.snap[i] = un;
    if (i == 1) {
      a.u_out[0] = T(1);
      if (a.snap) a.snap[0] = T(1);
    }
    if (i == a.nx - 2) {
      a.u_out[a.nx - 1] = T(1);
      if (a.snap) a.snap[a.nx - 1] = T(1);
    }
  }
}

template <typename T>
__global__ void k_fill_chi(T* u, int dim, int nx, int ny) {
  const int64_t J = (int64_t)nx * (dim == 2 ? ny : 1);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(j % nx);
    bool b = (i == 0 || i == nx - 1);
    if (dim == 2) {
      const int k = (int)(j / nx);
      b = b || k == 0 || k == ny - 1;
    }
    u[j] = b ? T(1) : T(0);
  }
}

__global__ void k_copy16(uint4* dst, const uint4* src, int64_t n16) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n16;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src[j];
}

template <typename T, int Q, int MINB>
cudaError_t launch2d_q(const Step2D<T>& a, cudaStream_t s) {
  const size_t smem = fk_step2d_smem(a.lx, a.ly, a.lyr, (int)sizeof(T));
  dim3 grid((a.nx - 2 + 31) / 32, (a.ny - 2 + a.ty - 1) / a.ty);
  k_step2d<T, Q, MINB><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int Q, int MINB>
cudaError_t attr2d_q() {
  return cudaFuncSetAttribute(k_step2d<T, Q, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

// Register-budget variants per precision: FP32 {4, 3} CTAs/SM, FP64 {2}.
template <typename T, int Q>
cudaError_t launch2d_var(const Step2D<T>& a, cudaStream_t s) {
  if (sizeof(T) == 8) return launch2d_q<T, Q, 2>(a, s);
  return a.variant == 1 ? launch2d_q<T, Q, 3>(a, s) : launch2d_q<T, Q, 4>(a, s);
}
template <typename T, int Q>
cudaError_t attr2d_var() {
  if (sizeof(T) == 8) return attr2d_q<T, Q, 2>();
  cudaError_t e = attr2d_q<T, Q, 4>();
  return e != cudaSuccess ? e : attr2d_q<T, Q, 3>();
}

template <typename T, int Q>
cudaError_t launch1d_q(const Step1D<T>& a, cudaStream_t s) {
  const size_t smem = fk_step1d_smem(a.lx, (int)sizeof(T));
  dim3 grid((a.nx - 2 + a.tx - 1) / a.tx);
  k_step1d<T, Q><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int Q>
cudaError_t attr1d_q() {
  return cudaFuncSetAttribute(k_step1d<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

size_t fk_step2d_smem(int lx, int ly, int lyr, int elem) {
  return (size_t)lx * lyr * (6 * elem) + (size_t)3 * lx * ly * elem;
}

size_t fk_step1d_smem(int lx, int elem) { return (size_t)lx * (4 * elem) + (size_t)lx * elem; }

template <typename T>
cudaError_t fk_launch_step2d(const Step2D<T>& a, int q, cudaStream_t s) {
  switch (q) {
    case 1: return launch2d_var<T, 1>(a, s);
    case 2: return launch2d_var<T, 2>(a, s);
    case 3: return launch2d_var<T, 3>(a, s);
    case 4: return launch2d_var<T, 4>(a, s);
    case 5: return launch2d_var<T, 5>(a, s);
    case 6: return launch2d_var<T, 6>(a, s);
    case 7: return launch2d_var<T, 7>(a, s);
    case 8: return launch2d_var<T, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t fk_launch_step1d(const Step1D<T>& a, int q, cudaStream_t s) {
  switch (q) {
    case 1: return launch1d_q<T, 1>(a, s);
    case 2: return launch1d_q<T, 2>(a, s);
    case 3: return launch1d_q<T, 3>(a, s);
    case 4: return launch1d_q<T, 4>(a, s);
    case 5: return launch1d_q<T, 5>(a, s);
    case 6: return launch1d_q<T, 6>(a, s);
    case 7: return launch1d_q<T, 7>(a, s);
    case 8: return launch1d_q<T, 8>(a, s);
    case 9: return launch1d_q<T, 9>(a, s);
    case 10: return launch1d_q<T, 10>(a, s);
    case 11: return launch1d_q<T, 11>(a, s);
    case 12: return launch1d_q<T, 12>(a, s);
    case 13: return launch1d_q<T, 13>(a, s);
    case 14: return launch1d_q<T, 14>(a, s);
    case 15: return launch1d_q<T, 15>(a, s);
    case 16: return launch1d_q<T, 16>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fk_prepare_step_kernels(int dim, int q, int elem) {
  if (dim == 2) {
    switch (q) {
#define FK_CASE(Q) \
  case Q: return elem == 4 ? attr2d_var<float, Q>() : attr2d_var<double, Q>();
      FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
#undef FK_CASE
      default: return cudaErrorInvalidValue;
    }
  }
  switch (q) {
#define FK_CASE(Q) \
  case Q: return elem == 4 ? attr1d_q<float, Q>() : attr1d_q<double, Q>();
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
    FK_CASE(9) FK_CASE(10) FK_CASE(11) FK_CASE(12) FK_CASE(13) FK_CASE(14) FK_CASE(15) FK_CASE(16)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t fk_launch_step2d<float>(const Step2D<float>&, int, cudaStream_t);
template cudaError_t fk_launch_step2d<double>(const Step2D<double>&, int, cudaStream_t);
template cudaError_t fk_launch_step1d<float>(const Step1D<float>&, int, cudaStream_t);
template cudaError_t fk_launch_step1d<double>(const Step1D<double>&, int, cudaStream_t);

cudaError_t fk_launch_fill_chi(void* u, int dim, int nx, int ny, int elem, cudaStream_t s) {
  const int64_t J = (int64_t)nx * (dim == 2 ? ny : 1);
  int blocks = (int)((J + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (elem == 4)
    k_fill_chi<float><<<blocks, 256, 0, s>>>((float*)u, dim, nx, ny);
  else
    k_fill_chi<double><<<blocks, 256, 0, s>>>((double*)u, dim, nx, ny);
  return cudaGetLastError();
}

cudaError_t fk_launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s) {
  if (bytes % 16 == 0 && ((uintptr_t)dst % 16) == 0 && ((uintptr_t)src % 16) == 0) {
    const int64_t n16 = bytes / 16;
    int blocks = (int)((n16 + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_copy16<<<blocks, 256, 0, s>>>((uint4*)dst, (const uint4*)src, n16);
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDeviceToDevice, s);
}
