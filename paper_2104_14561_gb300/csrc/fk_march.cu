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
#include "fk_device.cuh"

namespace {

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

template <typename T>
__device__ __forceinline__ T slope_fast(const T* u, int l, int stride, int g, int n) {
  if (g < 0 || g >= n) return T(0);
  const T* c = u + l * stride;
  if (g == 0) return pchip_fast(c[stride] - c[0], c[2 * stride] - c[stride]);
  if (g == n - 1) return pchip_fast(c[0] - c[-stride], c[-stride] - c[-2 * stride]);
  return pchip_fast(c[0] - c[-stride], c[stride] - c[0]);
}

// The same slope on a non-uniform mesh (raw derivative, not scaled): Eq.
// (e300) with the divided differences over the actual spacings x.
template <typename T>
__device__ __forceinline__ T slope_nu(const T* u, const T* x, int l, int stride, int g, int n) {
  if (g < 0 || g >= n) return T(0);
  auto del = [&](int m) { return (u[(m + 1) * stride] - u[m * stride]) / (x[m + 1] - x[m]); };
  if (g == 0) return pchip_fast(del(l), del(l + 1));
  if (g == n - 1) return pchip_fast(del(l - 1), del(l - 2));
  return pchip_fast(del(l - 1), del(l));
}

// Largest local index c in [1, hi] with x[c] <= z (bisection; x increasing).
template <typename T>
__device__ __forceinline__ int cell_of(const T* x, int hi, T z) {
  int lo = 1, up = hi + 1;
  while (up - lo > 1) {
    const int m = (lo + up) >> 1;
    if (x[m] <= z) lo = m; else up = m;
  }
  return lo;
}

// Record loads with explicit 32-bit shared-memory byte addresses: one add per
// query for the R and one for the S record, the second row at an immediate
// offset.  The compute phase only reads shared memory (it is written before
// the last __syncthreads), so the loads carry no ordering constraint.
__device__ __forceinline__ void lds_rec(uint32_t a, float& x, float& y, float& z, float& w) {
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
}
__device__ __forceinline__ void lds_rec_next(uint32_t a, float& x, float& y, float& z, float& w) {
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+16];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
}
__device__ __forceinline__ void lds_s(uint32_t a, float& x, float& y) {
  asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
}
__device__ __forceinline__ void lds_s_next(uint32_t a, float& x, float& y) {
  asm("ld.shared.v2.f32 {%0, %1}, [%2+8];" : "=f"(x), "=f"(y) : "r"(a));
}
__device__ __forceinline__ void lds_rec(uint32_t a, double& x, double& y, double& z, double& w) {
  asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a));
  asm("ld.shared.v2.f64 {%0, %1}, [%2+16];" : "=d"(z), "=d"(w) : "r"(a));
}
__device__ __forceinline__ void lds_rec_next(uint32_t a, double& x, double& y, double& z, double& w) {
  asm("ld.shared.v2.f64 {%0, %1}, [%2+32];" : "=d"(x), "=d"(y) : "r"(a));
  asm("ld.shared.v2.f64 {%0, %1}, [%2+48];" : "=d"(z), "=d"(w) : "r"(a));
}
__device__ __forceinline__ void lds_s(uint32_t a, double& x, double& y) {
  asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a));
}
__device__ __forceinline__ void lds_s_next(uint32_t a, double& x, double& y) {
  asm("ld.shared.v2.f64 {%0, %1}, [%2+16];" : "=d"(x), "=d"(y) : "r"(a));
}

// MINB = CTAs of 256 threads per SM that the register budget is sized for
// (4 -> <= 64 registers, 3 -> <= 85, 2 -> <= 128); the plan's autotuner
// picks the variant together with the tile height.

// Tiles are 32 nodes wide (one warp per tile row) and a multiple of 8 rows
// high (ty = 8 * passes); every staging loop walks rows by warp and columns
// by lane, so no index needs an integer division.
// Phases 1-3 of a step CTA: stage u^{n+1} over the tile plus halo, compute
// the scaled PCHIP slopes, pack the cell records.  gi0/gk0 are the global
// node indices of staged column / row 0.
// PX: periodic x (staged columns wrap modulo nx - 1; every x slope is an
// interior one).  NU: non-uniform mesh (the staged node coordinates go to
// SX, SY; the records hold raw derivatives, scaled per cell at the query).
template <bool MF, bool PX, bool NU, typename T>
__device__ __forceinline__ void stage_tile(const Step2D<T>& a, V4<T>* R, V2<T>* S, T* U, int gi0,
                                           int gk0, int warp, int lane) {
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  T* DX = U + lx * ly;
  T* DY = DX + lx * ly;
  T* SX = DY + lx * ly;
  T* SY = SX + lx;
  if constexpr (NU) {
    // coordinates of the staged nodes; outside the mesh far-away sentinels
    // (no point of an interior node lies there)
    for (int e = threadIdx.x; e < lx + ly; e += FK_THREADS) {
      if (e < lx) {
        const int gi = gi0 + e;
        SX[e] = gi < 0 ? T(-1e30) : (gi >= a.nx ? T(1e30) : a.xc[gi]);
      } else {
        const int gk = gk0 + e - lx;
        SY[e - lx] = gk < 0 ? T(-1e30) : (gk >= a.ny ? T(1e30) : a.yc[gk]);
      }
    }
  }
  // 1. stage u^{n+1} with asynchronous copies, all in flight at once (zero
  // fill outside the mesh; those entries are never read)
  const uint32_t sU = (uint32_t)__cvta_generic_to_shared(U);
  for (int lk = warp; lk < ly; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const bool rowin = gk >= 0 && gk < a.ny;
    const T* src = field_in<MF>(a) + (int64_t)(rowin ? gk : 0) * a.nx;
    for (int li = lane; li < lx; li += 32) {
      int gi = gi0 + li;
      if constexpr (PX) gi += gi < 0 ? a.nx - 1 : (gi >= a.nx - 1 ? 1 - a.nx : 0);
      const bool in = rowin && gi >= 0 && gi < a.nx;
      const T* g = in ? src + gi : field_in<MF>(a);
      const uint32_t d = sU + (uint32_t)(lk * lx + li) * (uint32_t)sizeof(T);
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(g),
                   "n"(sizeof(T)), "r"(in ? (int)sizeof(T) : 0));
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // 2. scaled PCHIP slopes h u_x, h u_y of the staged nodes 1..lx-2, 1..ly-2
  for (int lk = 1 + warp; lk <= ly - 2; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const T* row = U + lk * lx;
    for (int li = 1 + lane; li <= lx - 2; li += 32) {
      if constexpr (NU) {
        DX[lk * lx + li] = slope_nu(row, SX, li, 1, gi0 + li, a.nx);
        DY[lk * lx + li] = slope_nu(U + li, SY, lk, lx, gk, a.ny);
        continue;
      }
      if constexpr (PX)
        DX[lk * lx + li] = pchip_fast(row[li] - row[li - 1], row[li + 1] - row[li]);
      else
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
}

// The direct kernel.  mode 0: all interior rows.  mode 1: only the two row
// bands next to the y faces, [1, row_lo) and [row_hi, ny-1), whose shifted
// points may leave the box (the rows between go to the window kernel).
// Phase 4 of the direct kernel: the Gauss-Hermite sum of every output node
// of rows [k0, min(k0 + ty, k_end)) of this tile, one node per thread and
// pass (column i0 + lane, row k0 + warp + 8 m).  Returns the range-check flag.
template <typename T, int Q, bool MF, bool PX, bool NU>
__device__ __forceinline__ unsigned direct_phase(const Step2D<T>& a, const V4<T>* R,
                                                 const V2<T>* S, const T* SX, const T* SY,
                                                 int i0, int k0, int k_end, int gi0, int gk0,
                                                 int warp, int lane) {
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  const int i = i0 + lane;
  const int li = i - gi0;
  // periodic x: nodes 1 .. nx-1 (node 0 is node nx-1)
  const bool colok = i <= a.nx - (PX ? 1 : 2);
  T cx0 = T(0), cx1 = T(0), cx2 = T(0), cx3 = T(0);
  if (a.family == FK_CELLULAR_FLOW && colok) {
    const T* ct = a.col_tab + 4 * (int64_t)i;
    cx0 = ct[0]; cx1 = ct[1]; cx2 = ct[2]; cx3 = ct[3];
  }
  // the box relative to the node: in cells, or (NU) in physical lengths
  T nlo_x = T(-i), nhi_x = T(a.nx - 1 - i), xi = T(0);
  if constexpr (NU) {
    xi = SX[li];
    nlo_x = a.blo[0] - xi;
    nhi_x = a.bhi[0] - xi;
  }
  const uint32_t sR = (uint32_t)__cvta_generic_to_shared(R);
  const uint32_t sS = (uint32_t)__cvta_generic_to_shared(S);
  unsigned bad = 0;
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (!colok || k >= k_end) continue;
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
    T nlo_y = T(-k), nhi_y = T(a.ny - 1 - k), yk = T(0);
    if constexpr (NU) {
      yk = SY[lk];
      nlo_y = a.blo[1] - yk;
      nhi_y = a.bhi[1] - yk;
    }
    uint32_t rq[Q];  // byte offset of the query's lower row within a column of records
    T w0[Q], w1[Q], w2[Q], w3[Q];
    T exit_y = T(0);
    // NU: the points are sorted (ascending abscissae), so their cells are
    // too: bisect for the first, walk forward for the others
    int lcy = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T d = dy + a.gy[q];
      const bool out = (d < nlo_y) || (d > nhi_y);
      int lc;
      T t, hr = T(1);  // hr: the cell's height (NU), the slope basis scale
      if constexpr (NU) {
        const T z = yk + d;
        if (q == 0) {
          lcy = cell_of(SY, ly - 3, z);
        } else {
          while (lcy < ly - 3 && SY[lcy + 1] <= z) ++lcy;
        }
        lc = lcy;
        if (lc + gk0 > a.ny - 2) {
          lc = a.ny - 2 - gk0;
          t = T(1);
        } else {
          t = (z - SY[lc]) / (SY[lc + 1] - SY[lc]);
        }
        hr = SY[lc + 1] - SY[lc];
        if (!(t >= T(0) && t <= T(1))) {
          bad |= out ? 0u : 1u;
          t = T(0);
        }
      } else {
        const T fl = floor(d);
        int c = k + (int)fl;
        t = d - fl;
        if (c > a.ny - 2) {
          c = a.ny - 2;
          t = T(1);
        }
        lc = c - gk0;
      }
      if ((unsigned)(lc - 1) > (unsigned)(ly - 4)) {
        bad |= out ? 0u : 1u;
        lc = lk;
      }
      const T wq = out ? T(0) : a.w[q];
      exit_y += a.w[q] - wq;
      rq[q] = (uint32_t)(out ? lk : lc) * (uint32_t)sizeof(V2<T>);  // S stride; R stride is 2x
      const T t2 = t * t, omt = T(1) - t;
      w0[q] = wq;
      w1[q] = wq * (t2 * (T(3) - T(2) * t));  // h01
      w2[q] = wq * (t * omt * omt);            // h10
      w3[q] = -wq * (t2 * omt);                // h11
      if constexpr (NU) {
        w2[q] *= hr;
        w3[q] *= hr;
      }
    }
    const T om = T(1) - uj;
    T acc = T(0);
    int lcx = 0;  // NU: the cell of the previous x-point (0: none yet)
#pragma unroll 1
    for (int p = 0; p < Q; ++p) {
      const T d = dx + a.gx[p];
      if (!PX && ((d < nlo_x) || (d > nhi_x))) {
        acc += a.w[p] * om;
        continue;
      }
      int lc;
      T t, hc = T(1);  // hc: the cell's width (NU), the slope basis scale
      if constexpr (NU) {
        const T z = xi + d;
        if (lcx == 0) {
          lcx = cell_of(SX, lx - 3, z);
        } else {
          while (lcx < lx - 3 && SX[lcx + 1] <= z) ++lcx;
        }
        lc = lcx;
        if (lc + gi0 > a.nx - 2) {
          lc = a.nx - 2 - gi0;
          t = T(1);
        } else {
          t = (z - SX[lc]) / (SX[lc + 1] - SX[lc]);
        }
        hc = SX[lc + 1] - SX[lc];
        if (!(t >= T(0) && t <= T(1))) {
          bad |= 1u;
          t = T(0);
        }
      } else {
        const T fl = floor(d);
        int c = i + (int)fl;
        t = d - fl;
        if (!PX && c > a.nx - 2) {
          c = a.nx - 2;
          t = T(1);
        }
        lc = c - gi0;
      }
      if ((unsigned)(lc - 1) > (unsigned)(lx - 4)) {
        bad |= 1u;
        lc = li;
      }
      const T t2 = t * t, omt = T(1) - t;
      const T h01 = t2 * (T(3) - T(2) * t);
      const T h10 = t * omt * omt * hc, h11 = -(t2 * omt) * hc;
      const uint32_t baseS = sS + (uint32_t)(lc * lyr) * (uint32_t)sizeof(V2<T>);
      const uint32_t baseR = sR + (uint32_t)(lc * lyr) * (uint32_t)sizeof(V4<T>);
      T accp = exit_y * om;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        V4<T> r0, r1;
        V2<T> s0, s1;
        const uint32_t aR = baseR + 2 * rq[q], aS = baseS + rq[q];
        lds_rec(aR, r0.x, r0.y, r0.z, r0.w);
        lds_rec_next(aR, r1.x, r1.y, r1.z, r1.w);
        lds_s(aS, s0.x, s0.y);
        lds_s_next(aS, s1.x, s1.y);
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
    const int64_t j = (int64_t)k * a.nx + i;
    field_out<MF>(a)[j] = un;
    if (a.snap) a.snap[j] = un;
    if constexpr (PX) {
      write_periodic_x<MF>(a, i, k, un);
    } else {
      write_adjacent_boundary<MF>(a, i, k);
    }
  }
  return bad;
}

// MF: several fields per launch (blockIdx.z), for Algorithm 1.  PX:
// periodic x.  NU: non-uniform mesh.
template <typename T, int Q, int MINB, bool MF, bool PX, bool NU>
__global__ void __launch_bounds__(FK_THREADS, MINB) k_step2d(const Step2D<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  V2<T>* S = reinterpret_cast<V2<T>*>(R + lx * lyr);
  T* U = reinterpret_cast<T*>(S + lx * lyr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int i0 = 1 + blockIdx.x * 32;  // first interior output node of the tile
  int k0, k_end;
  if (a.mode == 0) {
    k0 = 1 + blockIdx.y * a.ty;
    k_end = a.ny - 1;
  } else if ((int)blockIdx.y < a.nb_lo) {
    k0 = 1 + blockIdx.y * a.ty;
    k_end = a.row_lo;
  } else {
    k0 = a.row_hi + (blockIdx.y - a.nb_lo) * a.ty;
    k_end = a.ny - 1;
  }
  const int gi0 = i0 - a.hx - 1;  // global node of staged column 0
  const int gk0 = k0 - a.hy - 1;
  stage_tile<MF, PX, NU>(a, R, S, U, gi0, gk0, warp, lane);
  const T* SX = U + 3 * lx * ly;  // staged coordinates (NU)
  const T* SY = SX + lx;
  const unsigned bad =
      direct_phase<T, Q, MF, PX, NU>(a, R, S, SX, SY, i0, k0, k_end, gi0, gk0, warp, lane);
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// Record loads at a compile-time row offset from a per-x-point base address.
template <int OFF>
__device__ __forceinline__ void lds_rec_at(uint32_t a, float& x, float& y, float& z, float& w) {
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
      : "=f"(x), "=f"(y), "=f"(z), "=f"(w)
      : "r"(a), "n"(OFF));
}
template <int OFF>
__device__ __forceinline__ void lds_s_at(uint32_t a, float& x, float& y) {
  asm("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(x), "=f"(y) : "r"(a), "n"(OFF));
}

template <int W, int R>
struct WinRows {
  // acc += sum over rows r >= R of Phi_r (row value - u_j) + Psi_r (row slope)
  __device__ __forceinline__ static void run(uint32_t aR, uint32_t aS, float uj, float h01,
                                             float h10, float h11, const float* phi,
                                             const float* psi, float& acc0, float& acc1) {
    float4 r;
    float2 s;
    lds_rec_at<16 * R>(aR, r.x, r.y, r.z, r.w);
    lds_s_at<8 * R>(aS, s.x, s.y);
    const float rb = (r.x - uj) + h01 * r.y + h10 * r.z + h11 * r.w;
    const float sb = s.x + h01 * s.y;
    acc0 += phi[R] * rb;
    acc1 += psi[R] * sb;
    WinRows<W, R + 1>::run(aR, aS, uj, h01, h10, h11, phi, psi, acc0, acc1);
  }
};
template <int W>
struct WinRows<W, W> {
  __device__ __forceinline__ static void run(uint32_t, uint32_t, float, float, float, float,
                                             const float*, const float*, float&, float&) {}
};

// Adds (v0, v1, v2) to rows (m, m+1, m+2) of a register window; m is the
// same for every thread of the launch (a plan constant), so the switch is a
// uniform branch and the window stays in registers.
template <int W, int M>
struct WinAdd {
  __device__ __forceinline__ static void run(int m, float* f, float v0, float v1, float v2) {
    if (m == M) {
      f[M] += v0;
      f[M + 1] += v1;
      f[M + 2] += v2;
    } else {
      WinAdd<W, M + 1>::run(m, f, v0, v1, v2);
    }
  }
};
template <int W>
struct WinAdd<W, W - 2> {
  __device__ __forceinline__ static void run(int, float*, float, float, float) {}
};

// The window kernel (FP32), for interior rows [row_lo, row_hi) whose
// shifted points all stay strictly inside the box along y.  Per node the
// y-points q of the tensor rule fall in cells c_q = c_0 + o_q with
// o_q = m_q + beta_q, m_q = floor(gy_q - gy_0) a plan constant and
// beta_q in {0, 1}; the sum over q of the y-Hermite weights is collected
// per cell row into Phi_r (value basis) and Psi_r (slope basis), r < W.
// Then for every x-point p each of the W rows is read once (24 bytes) and
//   sum_q w_q (Itilde(x_p, y_q) - u_j) = sum_r Phi_r (row_r(x_p) - u_j)
//                                            + Psi_r slope_r(x_p),
// exactly the direct form's sum (zero-twist bicubic: Itilde is linear in
// the row values, and sum_r Phi_r = sum_q w_q = 1), with W row reads
// instead of 2Q per x-point.
template <int Q, int W>
__global__ void __launch_bounds__(FK_THREADS, 4) k_step2dw(const Step2D<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using T = float;
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  V2<T>* S = reinterpret_cast<V2<T>*>(R + lx * lyr);
  T* U = reinterpret_cast<T*>(S + lx * lyr);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = 1 + blockIdx.x * 32;
  // tiles [0, nwin) cover the window rows; the rest cover the two bands
  // next to the y faces with the direct path (one launch per step)
  const int nwin = (a.row_hi - a.row_lo + a.ty - 1) / a.ty;
  const bool window = (int)blockIdx.y < nwin;
  int k0, k_end;
  if (window) {
    k0 = a.row_lo + blockIdx.y * a.ty;
    k_end = a.row_hi;
  } else if ((int)blockIdx.y - nwin < a.nb_lo) {
    k0 = 1 + (blockIdx.y - nwin) * a.ty;
    k_end = a.row_lo;
  } else {
    k0 = a.row_hi + (blockIdx.y - nwin - a.nb_lo) * a.ty;
    k_end = a.ny - 1;
  }
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;
  stage_tile<false, false, false>(a, R, S, U, gi0, gk0, warp, lane);
  if (!window) {
    const unsigned b = direct_phase<T, Q, false, false, false>(a, R, S, nullptr, nullptr, i0, k0,
                                                               k_end, gi0, gk0, warp, lane);
    if (b) atomicOr(a.err, FK_DEVERR_RANGE);
    return;
  }

  const int i = i0 + lane;
  const int li = i - gi0;
  const bool colok = i <= a.nx - 2;
  T cx0 = T(0), cx1 = T(0), cx2 = T(0), cx3 = T(0);
  if (a.family == FK_CELLULAR_FLOW && colok) {
    const T* ct = a.col_tab + 4 * (int64_t)i;
    cx0 = ct[0]; cx1 = ct[1]; cx2 = ct[2]; cx3 = ct[3];
  }
  const T nlo_x = T(-i), nhi_x = T(a.nx - 1 - i);
  const uint32_t sR = (uint32_t)__cvta_generic_to_shared(R);
  const uint32_t sS = (uint32_t)__cvta_generic_to_shared(S);
  unsigned bad = 0;
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (!colok || k >= a.row_hi) continue;
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
    // y window: rows c_0 .. c_0 + W - 1 relative to the staged tile
    const int c0 = (int)floor(dy + a.gy[0]);
    int lrow0 = k + c0 - gk0;
    if (lrow0 < 1 || lrow0 + W - 1 > ly - 2) {
      bad |= 1u;
      lrow0 = 1;
    }
    T phi[W], psi[W];
#pragma unroll
    for (int r = 0; r < W; ++r) {
      phi[r] = T(0);
      psi[r] = T(0);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T d = dy + a.gy[q];
      const T fl = floor(d);
      const T t = d - fl;
      const int beta = (int)fl - c0 - a.wm[q];
      if ((unsigned)beta > 1u) bad |= 1u;
      const T t2 = t * t, omt = T(1) - t;
      const T wq = a.w[q];
      const T w01 = wq * (t2 * (T(3) - T(2) * t)), w00 = wq - w01;
      const T w10 = wq * (t * omt * omt), w11 = -wq * (t2 * omt);
      const bool b1 = beta == 1;
      WinAdd<W, 0>::run(a.wm[q], phi, b1 ? T(0) : w00, b1 ? w00 : w01, b1 ? w01 : T(0));
      WinAdd<W, 0>::run(a.wm[q], psi, b1 ? T(0) : w10, b1 ? w10 : w11, b1 ? w11 : T(0));
    }
    const T om = T(1) - uj;
    const uint32_t rowR = (uint32_t)lrow0 * (uint32_t)sizeof(V4<T>);
    const uint32_t rowS = (uint32_t)lrow0 * (uint32_t)sizeof(V2<T>);
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
      const uint32_t colR = sR + (uint32_t)(lc * lyr) * (uint32_t)sizeof(V4<T>) + rowR;
      const uint32_t colS = sS + (uint32_t)(lc * lyr) * (uint32_t)sizeof(V2<T>) + rowS;
      T acc0 = T(0), acc1 = T(0);
      WinRows<W, 0>::run(colR, colS, uj, h01, h10, h11, phi, psi, acc0, acc1);
      acc += a.w[p] * (acc0 + acc1);
    }
    const T un = uj + acc;
    const int64_t j = (int64_t)k * a.nx + i;
    a.u_out[j] = un;
    if (a.snap) a.snap[j] = un;
    write_adjacent_boundary<false>(a, i, k);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// 1D step: same structure with a record {u_c, u_{c+1}-u_c, h u'_c, h u'_{c+1}}
// per staged cell.  NU: non-uniform mesh (staged coordinates SX, raw
// derivatives in the records, cell search, per-cell widths), as in 2D.
template <typename T, int Q, bool NU>
__global__ void __launch_bounds__(FK_THREADS) k_step1d(const Step1D<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  T* U = reinterpret_cast<T*>(R + lx);
  T* SX = U + lx;  // NU only
  const int i0 = 1 + blockIdx.x * a.tx;
  const int gi0 = i0 - a.hx - 1;
  const T* const uin = a.in();
  T* const uo = a.out();
  for (int e = threadIdx.x; e < lx; e += blockDim.x) {
    const int gi = gi0 + e;
    U[e] = (gi >= 0 && gi < a.nx) ? uin[gi] : T(0);
    if constexpr (NU) SX[e] = gi < 0 ? T(-1e30) : (gi >= a.nx ? T(1e30) : a.xc[gi]);
  }
  __syncthreads();
  for (int lc = 1 + threadIdx.x; lc <= lx - 3; lc += blockDim.x) {
    const int gi = gi0 + lc;
    V4<T> r;
    r.x = U[lc];
    r.y = U[lc + 1] - U[lc];
    if constexpr (NU) {
      r.z = slope_nu(U, SX, lc, 1, gi, a.nx);
      r.w = slope_nu(U, SX, lc + 1, 1, gi + 1, a.nx);
    } else {
      r.z = slope_line(U, lc, 1, gi, a.nx);
      r.w = slope_line(U, lc + 1, 1, gi + 1, a.nx);
    }
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
    int lcw = 0;  // NU: the cell of the previous point (the points are sorted)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int lc;
      T t, hc = T(1);  // hc: the cell's width (NU), the slope basis scale
      if constexpr (NU) {
        const T z = SX[li] + (a.cdx + a.g[q]);
        if (z < a.blo || z > a.bhi) {
          acc += a.w[q] * om;
          continue;
        }
        if (lcw == 0) {
          lcw = cell_of(SX, lx - 3, z);
        } else {
          while (lcw < lx - 3 && SX[lcw + 1] <= z) ++lcw;
        }
        lc = lcw;
        if (lc + gi0 > a.nx - 2) {
          lc = a.nx - 2 - gi0;
          t = T(1);
        } else {
          t = (z - SX[lc]) / (SX[lc + 1] - SX[lc]);
        }
        hc = SX[lc + 1] - SX[lc];
        if (!(t >= T(0) && t <= T(1))) {
          bad |= 1u;
          t = T(0);
        }
      } else {
        int c;
        const bool out = locate(i, a.cdx + a.g[q], a.nx, &c, &t);
        if (out) {
          acc += a.w[q] * om;
          continue;
        }
        lc = c - gi0;
      }
      if (lc < 1 || lc > lx - 3) {
        bad |= 1u;
        lc = li;
      }
      const T t2 = t * t, omt = T(1) - t;
      const V4<T> r = R[lc];
      const T v = (r.x - uj) + (t2 * (T(3) - T(2) * t)) * r.y + (t * omt * omt * hc) * r.z -
                  (t2 * omt * hc) * r.w;
      acc += a.w[q] * v;
    }
    if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
    const T un = uj + acc;
    uo[i] = un;
    if (a.snap) a.snap[i] = un;
    if (i == 1) {
      uo[0] = T(1);
      if (a.snap) a.snap[0] = T(1);
    }
    if (i == a.nx - 2) {
      uo[a.nx - 1] = T(1);
      if (a.snap) a.snap[a.nx - 1] = T(1);
    }
  }
}

// Whether flat node j lies on an absorbing face (Eq. (e3)); with px the x
// faces are identified and only the other faces count.
__device__ __forceinline__ bool on_boundary(int64_t j, int dim, int nx, int ny, int nz, int px) {
  const int i = (int)(j % nx);
  bool b = !px && (i == 0 || i == nx - 1);
  if (dim >= 2) {
    const int k = (int)((j / nx) % ny);
    b = b || k == 0 || k == ny - 1;
  }
  if (dim == 3) {
    const int l = (int)(j / ((int64_t)nx * ny));
    b = b || l == 0 || l == nz - 1;
  }
  return b;
}

template <typename T>
__global__ void k_fill_chi(T* u, int dim, int nx, int ny, int px, int nz) {
  const int64_t J = (int64_t)nx * (dim >= 2 ? ny : 1) * (dim == 3 ? nz : 1);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    u[j] = on_boundary(j, dim, nx, ny, nz, px) ? T(1) : T(0);
  }
}

template <typename T>
__global__ void k_fill_fields(T* even, T* odd, const T* src, int dim, int nx, int ny, int nf,
                              int px, int nz) {
  const int64_t J = (int64_t)nx * (dim >= 2 ? ny : 1) * (dim == 3 ? nz : 1), total = J * nf;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / J, j = e - c * J;  // field c + 1
    T v;
    if (src) {
      v = src[j];
    } else {
      v = on_boundary(j, dim, nx, ny, nz, px) ? T(1) : T(0);
    }
    (((c + 1) & 1) ? odd : even)[e] = v;
  }
}

__global__ void k_copy16(uint4* dst, const uint4* src, int64_t n16) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n16;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src[j];
}

// Register budget of the several-field launches: FP32 4 CTAs/SM, FP64 2.
template <typename T>
constexpr int kMinbFields = sizeof(T) == 8 ? 2 : 4;

template <typename T, int Q, int MINB>
cudaError_t launch2d_q(const Step2D<T>& a, cudaStream_t s) {
  const size_t smem = fk_step2d_smem(a.lx, a.ly, a.lyr, (int)sizeof(T), a.nu);
  int gy;
  if (a.mode == 0)
    gy = (a.ny - 2 + a.ty - 1) / a.ty;
  else
    gy = a.nb_lo + (a.ny - 1 - a.row_hi + a.ty - 1) / a.ty;
  if (gy <= 0) return cudaSuccess;
  const int nf = a.ncols > 1 ? a.ncols : 1;
  constexpr int D = kMinbFields<T>;
  if (a.px) {  // periodic x: nodes 1 .. nx-1, the default register budget
    dim3 grid((a.nx - 1 + 31) / 32, gy, nf);
    if (nf > 1)
      k_step2d<T, Q, D, true, true, false><<<grid, FK_THREADS, smem, s>>>(a);
    else
      k_step2d<T, Q, D, false, true, false><<<grid, FK_THREADS, smem, s>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((a.nx - 2 + 31) / 32, gy, nf);
  if (a.nu) {  // non-uniform mesh, the default register budget
    if (nf > 1)
      k_step2d<T, Q, D, true, false, true><<<grid, FK_THREADS, smem, s>>>(a);
    else
      k_step2d<T, Q, D, false, false, true><<<grid, FK_THREADS, smem, s>>>(a);
    return cudaGetLastError();
  }
  if (nf > 1)
    k_step2d<T, Q, D, true, false, false><<<grid, FK_THREADS, smem, s>>>(a);
  else
    k_step2d<T, Q, MINB, false, false, false><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// The window kernel stages one extra halo row in y: its window can reach
// one row past the cells the points use (a row of weight 0).
inline Step2D<float> window_args(const Step2D<float>& a) {
  Step2D<float> w = a;
  w.hy = a.hy + 1;
  w.ly = w.ty + 2 * w.hy + 2;
  w.lyr = w.ly | 1;
  return w;
}

template <int Q, int W>
cudaError_t launchw(const Step2D<float>& a, cudaStream_t s) {
  const Step2D<float> w = window_args(a);
  const size_t smem = fk_step2d_smem(w.lx, w.ly, w.lyr, 4);
  const int nwin = (w.row_hi - w.row_lo + w.ty - 1) / w.ty;
  const int nb_hi = (w.ny - 1 - w.row_hi + w.ty - 1) / w.ty;
  dim3 grid((w.nx - 2 + 31) / 32, nwin + w.nb_lo + nb_hi);
  k_step2dw<Q, W><<<grid, FK_THREADS, smem, s>>>(w);
  return cudaGetLastError();
}
template <int Q, int W>
cudaError_t attrw() {
  return cudaFuncSetAttribute(k_step2dw<Q, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

// (Q, W) pairs with a window kernel: Q in {4, 6, 8}, 3 <= W <= 2Q - 1.
#define FK_WIN_LIST(X)                                                                     \
  X(4, 3) X(4, 4) X(4, 5) X(4, 6) X(4, 7)                                                  \
  X(6, 3) X(6, 4) X(6, 5) X(6, 6) X(6, 7) X(6, 8) X(6, 9) X(6, 10) X(6, 11)                \
  X(8, 3) X(8, 4) X(8, 5) X(8, 6) X(8, 7) X(8, 8) X(8, 9) X(8, 10) X(8, 11) X(8, 12)       \
  X(8, 13) X(8, 14) X(8, 15)

cudaError_t launch_window(const Step2D<float>& a, int q, cudaStream_t s) {
#define FK_W(QQ, WW) \
  if (q == QQ && a.win == WW) return launchw<QQ, WW>(a, s);
  FK_WIN_LIST(FK_W)
#undef FK_W
  return cudaErrorInvalidValue;
}

template <typename T, int Q, int MINB>
cudaError_t attr2d_q() {
  const int big = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, false, false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if constexpr (MINB == kMinbFields<T>) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, true, false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, false, true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, true, true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, false, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step2d<T, Q, MINB, true, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  }
  return e;
}

// Register-budget variants per precision: FP32 {4, 3} CTAs/SM, FP64 {2}.
template <typename T, int Q>
cudaError_t launch2d_var(const Step2D<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    return launch2d_q<T, Q, 2>(a, s);
  } else {
    return a.variant == 1 ? launch2d_q<T, Q, 3>(a, s) : launch2d_q<T, Q, 4>(a, s);
  }
}
template <typename T, int Q>
cudaError_t attr2d_var() {
  if constexpr (sizeof(T) == 8) {
    return attr2d_q<T, Q, 2>();
  } else {
    cudaError_t e = attr2d_q<T, Q, 4>();
    return e != cudaSuccess ? e : attr2d_q<T, Q, 3>();
  }
}

template <typename T, int Q>
cudaError_t launch1d_q(const Step1D<T>& a, cudaStream_t s) {
  const size_t smem = fk_step1d_smem(a.lx, (int)sizeof(T), a.nu);
  dim3 grid((a.nx - 2 + a.tx - 1) / a.tx, 1, a.ncols > 1 ? a.ncols : 1);
  if (a.nu)
    k_step1d<T, Q, true><<<grid, FK_THREADS, smem, s>>>(a);
  else
    k_step1d<T, Q, false><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int Q>
cudaError_t attr1d_q() {
  cudaError_t e = cudaFuncSetAttribute(k_step1d<T, Q, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step1d<T, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
  return e;
}

}  // namespace

size_t fk_step2d_smem(int lx, int ly, int lyr, int elem, int nu) {
  return (size_t)lx * lyr * (6 * elem) + (size_t)3 * lx * ly * elem +
         (nu ? (size_t)(lx + ly) * elem : 0);
}

size_t fk_step1d_smem(int lx, int elem, int nu) {
  return (size_t)lx * (4 * elem) + (size_t)lx * elem + (nu ? (size_t)lx * elem : 0);
}

bool fk_window_available(int q, int w) {
#define FK_W(QQ, WW) \
  if (q == QQ && w == WW) return true;
  FK_WIN_LIST(FK_W)
#undef FK_W
  return false;
}

template <typename T>
cudaError_t fk_launch_step2d(const Step2D<T>& a, int q, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (a.mode == 2) return fk_launch_step2dm64(a, q, s);  // masked tensor window, FP64
  }
  if constexpr (sizeof(T) == 4) {
    if (a.mode == 2) return fk_launch_step2dm(a, q, s);  // masked tensor window
    if (a.win > 0) {
      if (a.ncols <= 1) return launch_window(a, q, s);  // window rows and face bands
      // several fields: the direct kernel on every row (same tile and halo)
      Step2D<float> d = a;
      d.win = 0;
      d.mode = 0;
      return fk_launch_step2d<float>(d, q, s);
    }
  }
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
  if (dim == 2 && elem == 8) {
    cudaError_t em = fk_prepare_masked64(q);
    if (em != cudaSuccess) return em;
  }
  if (dim == 2 && elem == 4) {
    cudaError_t em = fk_prepare_masked_kernels(q);
    if (em != cudaSuccess) return em;
#define FK_W(QQ, WW)                     \
  if (q == QQ) {                         \
    cudaError_t e = attrw<QQ, WW>();     \
    if (e != cudaSuccess) return e;      \
  }
    FK_WIN_LIST(FK_W)
#undef FK_W
  }
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

cudaError_t fk_launch_fill_chi(void* u, int dim, int nx, int ny, int elem, cudaStream_t s,
                               int px, int nz) {
  const int64_t J = (int64_t)nx * (dim >= 2 ? ny : 1) * (dim == 3 ? nz : 1);
  int blocks = (int)((J + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (elem == 4)
    k_fill_chi<float><<<blocks, 256, 0, s>>>((float*)u, dim, nx, ny, px, nz);
  else
    k_fill_chi<double><<<blocks, 256, 0, s>>>((double*)u, dim, nx, ny, px, nz);
  return cudaGetLastError();
}

cudaError_t fk_launch_fill_fields(void* even, void* odd, const void* src, int dim, int nx, int ny,
                                  int elem, int nfields, cudaStream_t s, int px, int nz) {
  const int64_t total = (int64_t)nx * (dim >= 2 ? ny : 1) * (dim == 3 ? nz : 1) * nfields;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (elem == 4)
    k_fill_fields<float><<<blocks, 256, 0, s>>>((float*)even, (float*)odd, (const float*)src, dim,
                                                nx, ny, nfields, px, nz);
  else
    k_fill_fields<double><<<blocks, 256, 0, s>>>((double*)even, (double*)odd,
                                                 (const double*)src, dim, nx, ny, nfields, px, nz);
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
