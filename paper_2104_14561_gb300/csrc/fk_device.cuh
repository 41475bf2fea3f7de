// Device helpers shared by the step kernels of libfk_gb300 (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fk_internal.h"

namespace {

// Packed FP32 pairs (two lanes of work per instruction on sm_100 and later).
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The fields of a step launch: with MF (several fields, Algorithm 1) the
// field of blockIdx.z, else u_in / u_out as passed (no offset arithmetic
// in the single-field kernels).
template <bool MF, typename T>
__device__ __forceinline__ const T* field_in(const Step2D<T>& a) {
  if constexpr (MF) return a.in();
  else return a.u_in;
}
template <bool MF, typename T>
__device__ __forceinline__ T* field_out(const Step2D<T>& a) {
  if constexpr (MF) return a.out();
  else return a.u_out;
}

// Values the compiler cannot see through.  An offset by opaque_zero()
// keeps per-point constants in shared memory from being hoisted out of a
// loop into registers held across it; opaque(x) makes a later use of x
// recompute what it derives from x instead of keeping those results live.
__device__ __forceinline__ int opaque_zero() {
  int z;
  asm volatile("mov.u32 %0, 0;" : "=r"(z));
  return z;
}
__device__ __forceinline__ float opaque(float x) {
  float y;
  asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Scaled PCHIP slope h*u'_j from the two neighbouring differences
// (Eq. (e300)): 0 unless both have the same strict sign, else their
// harmonic mean 2 dl dr / (dl + dr).
template <typename T>
__device__ __forceinline__ T pchip_scaled(T dl, T dr) {
  const T p = dl * dr;
  return p > T(0) ? (T(2) * p) / (dl + dr) : T(0);
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

// The FP32 slope of Eq. (e300) with the hardware reciprocal approximation
// (rcp.approx: relative error below 2^-22) times 2 p: the quotient is a
// few ulp, inside the FP32 parity budget like pchip_fast.  When p > 0 both
// differences have the same sign and are normal, so their sum is normal
// and flushing subnormal inputs changes nothing.
__device__ __forceinline__ float pchip_rcp(float dl, float dr) {
  const float p = dl * dr;
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(dl + dr));
  const float h = p * r;
  return p > 0.f ? h + h : 0.f;
}

// Boundary nodes adjacent to interior node (i, k) hold 1 (Eq. (e3)), in
// out (and snap when given).  On a mesh with 3 nodes along an axis the
// single interior line is next to both faces of that axis, so every flag is
// tested on its own.
template <typename T>
__device__ __forceinline__ void boundary_ones(T* out, T* snap, int nx_, int ny_, int i, int k) {
  const int64_t nx = nx_;
  const bool L = (i == 1), Rt = (i == nx_ - 2), B = (k == 1), Tp = (k == ny_ - 2);
  if (L | Rt | B | Tp) {
    const int64_t top = (int64_t)(ny_ - 1) * nx, row = (int64_t)k * nx;
    auto one = [&](int64_t j) {
      out[j] = T(1);
      if (snap) snap[j] = T(1);
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
template <bool MF, typename T>
__device__ __forceinline__ void write_adjacent_boundary(const Step2D<T>& a, int i, int k) {
  const int64_t nx = a.nx;
  const bool L = (i == 1), Rt = (i == a.nx - 2), B = (k == 1), Tp = (k == a.ny - 2);
  if (L | Rt | B | Tp) {
    const int64_t top = (int64_t)(a.ny - 1) * nx, row = (int64_t)k * nx;
    auto one = [&](int64_t j) {
      field_out<MF>(a)[j] = T(1);
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


// Periodic x: node (nx-1, k) is node (0, k), so it gets the same value;
// the y-face nodes of the column (and of column 0 with it) hold 1.
template <bool MF, typename T>
__device__ __forceinline__ void write_periodic_x(const Step2D<T>& a, int i, int k, T un) {
  const int64_t nx = a.nx, top = (int64_t)(a.ny - 1) * nx;
  const bool last = (i == a.nx - 1);
  auto put = [&](int64_t j, T v) {
    field_out<MF>(a)[j] = v;
    if (a.snap) a.snap[j] = v;
  };
  if (last) put((int64_t)k * nx, un);
  if (k == 1) {
    put(i, T(1));
    if (last) put(0, T(1));
  }
  if (k == a.ny - 2) {
    put(top + i, T(1));
    if (last) put(top, T(1));
  }
}

// Staging of the masked tensor-window kernels (the step and its adjoint),
// for a CTA of FK_THREADS threads whose staged node (0, 0) is global node
// (gi0, gk0); a.lx x a.ly nodes, row pitch a.lyr (odd).  Ends with the
// records visible to the whole CTA.
template <bool MF = false>
__device__ __forceinline__ void masked_stage(const Step2D<float>& a, float4* Rec, float* U,
                                             int gi0, int gk0) {
  const int lx = a.lx, ly = a.ly, lp = a.lyr;
  const int tid = threadIdx.x;
  // 1. u^{n+1} over the tile and halo, row-major with pitch lp (zero
  // outside the mesh): rows by warp, columns by lane, so global reads are
  // coalesced and shared-memory writes consecutive
  {
    const uint32_t sU = (uint32_t)__cvta_generic_to_shared(U);
    const int lane = tid & 31, warp = tid >> 5;
    for (int r = warp; r < ly; r += FK_THREADS / 32) {
      const int gk = gk0 + r;
      const bool rowin = (unsigned)gk < (unsigned)a.ny;
      const float* src = field_in<MF>(a) + (int64_t)(rowin ? gk : 0) * a.nx;
      const uint32_t drow = sU + (uint32_t)(r * lp) * 4u;
      for (int c = lane; c < lx; c += 32) {
        const int gi = gi0 + c;
        const bool in = rowin && (unsigned)gi < (unsigned)a.nx;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(drow + 4u * c),
                     "l"(in ? src + gi : field_in<MF>(a)), "r"(in ? 4 : 0));
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
  }

  // 2. records {u, h u_x, h u_y, 0} of staged nodes 1..lx-2 x 1..ly-2, by
  // vertical sweeps: thread t owns column 1 + t % hc and a segment of rows,
  // carrying u of the rows above and below in registers.  The end rule
  // stated after Eq. (e300) gives node 0 the slope of node 1 and node n-1
  // that of node n-2 (the harmonic mean is symmetric): an end column takes
  // its x-differences one column inwards, and the end rows copy the y-slope
  // of their neighbour row afterwards.  Nodes outside the mesh get finite
  // values from the zero fill; they only ever carry weight 0.
  {
    const int hc = lx - 2, hr = ly - 2;
    const int nseg = FK_THREADS / hc;  // hc <= 256: lx <= 258
    const int seg = tid / hc, c = 1 + (tid - seg * hc);
    if (seg < nseg) {
      const int len = (hr + nseg - 1) / nseg;
      const int r0 = 1 + seg * len, r1 = min(r0 + len, hr + 1);
      const int gi = gi0 + c;
      const int ax = c + (gi == 0) - (gi == a.nx - 1);
      const float* col = U + c;
      const float* colx = U + ax;
      float up = col[(r0 - 1) * lp], uc = col[r0 * lp];
      for (int r = r0; r < r1; ++r) {
        const float un = col[(r + 1) * lp];
        const float* rx = colx + r * lp;
        const float X = pchip_fast(rx[0] - rx[-1], rx[1] - rx[0]);
        const float Y = pchip_fast(uc - up, un - uc);
        Rec[r * lp + c] = make_float4(uc, X, Y, 0.f);
        up = uc;
        uc = un;
      }
    }
    __syncthreads();
    // y end rule: staged rows of mesh rows 0 and ny-1 take their neighbour's y-slope
    const int rb = -gk0, rt = a.ny - 1 - gk0;
    const bool fb = rb >= 1 && rb <= hr, ft = rt >= 1 && rt <= hr;
    if (fb || ft) {
      for (int e = tid; e < hc; e += FK_THREADS) {
        if (fb) Rec[rb * lp + 1 + e].z = Rec[(rb + 1) * lp + 1 + e].z;
        if (ft) Rec[rt * lp + 1 + e].z = Rec[(rt - 1) * lp + 1 + e].z;
      }
      __syncthreads();
    }
  }

}

}  // namespace
