// Device helpers shared by the step kernels of libfk_gb300 (internal).
#pragma once

#include <cuda_runtime.h>
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

// Boundary nodes adjacent to interior node (i, k) hold 1 (Eq. (e3)).  On a
// mesh with 3 nodes along an axis the single interior line is next to both
// faces of that axis, so every flag is tested on its own.
template <typename T>
__device__ __forceinline__ void write_adjacent_boundary(const Step2D<T>& a, int i, int k) {
  const int64_t nx = a.nx;
  const bool L = (i == 1), Rt = (i == a.nx - 2), B = (k == 1), Tp = (k == a.ny - 2);
  if (L | Rt | B | Tp) {
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

}  // namespace
