// Adjoint of the march: dL/dtheta and dL/du^N for L = <g, u^0>.
//
// Step n of Scheme 1 maps u^{n+1} to u^n through the slope map F
// (Eq. (e300)), the interpolation at the shifted points (Eq. (e34)) and the
// quadrature (Eq. (e35)): u^n = A_n [u^{n+1}; F(u^{n+1})] + c_n
// (Eq. (e36)).  Going backward, with lambda^n = dL/du^n:
//   mu            = A_n^T lambda^n          (k_adj_scatter: per query, the
//                   12 interpolation weights scattered to the cell corners,
//                   shared-memory atomics within a tile, global atomics for
//                   the tile's halo),
//   lambda^{n+1}  = mu_u + dF^T mu_D         (k_adj_slopes_t: a gather over
//                   the 3-node slope stencil and the end rule),
//   dL/dtheta    += lambda^n . dS_n/dtheta   (k_adj_scatter: the spatial
//                   derivative of the interpolant at each shifted point
//                   times the shifted point's derivative in (A, eps, omega,
//                   D) or (b_1, b_2, -, s); FP64 reduction over nodes).
// The exit value 1 and the boundary rows depend on nothing.  The slope
// rule is differentiated on its active branch (0 on the zero branch).
//
// Memory: u is checkpointed every K steps on a forward pass; each segment
// of K steps is recomputed from its checkpoint before its backward steps.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {

template <typename T>
struct AdjArgs {
  Step2D<T> s;      // u_in = u^{n+1}; staging and drift as in the forward step
  const T* lam;     // lambda^n, or nullptr: the masked kernel forms it (below)
  T* mu;            // 3 J accumulators (zero on entry): [u; h u_x; h u_y] parts
  // lam == nullptr (masked form): lambda^n at the tile's nodes is the
  // slope transpose of the previous backward step's accumulators mu_prev
  // over u_prev, the field whose slopes that step took; the kernel also
  // zeroes mu_clear at its nodes (and the boundary nodes next to them),
  // the accumulators of the step after this one
  const T* mu_prev;
  const T* u_prev;
  T* mu_clear;
  double* dth;      // 4 parameter derivatives (accumulated)
  // d(shift in cells)/d theta_k = ax_k + cn_k g (x) and ay_k + cn_k g (y):
  // cellular flow: ax_A = kx cy sx1, ax_eps = kx cy st sx2, ax_om = kx cy sw sx2
  //                (and 2 st, 2 sw with cx2 for y); constant drift: ax_b1 = dt/hx
  T st, sw;         // sin(omega t_n), eps t_n cos(omega t_n)
  T cbx, cby;       // constant drift: dt / h per axis
  T cn;             // d sigma / d theta_3 divided by sigma
  // masked form, nodes whose points all stay inside: the 1D weights as
  // piecewise cubics in the fractional cell position of point 0
  const float4* tab;          // see adj_tables
  float brk[2][FK_MAXQ_2D];   // piece boundaries per axis, unused ones 2
  float last[2];              // g_{Q-1} - g_0 per axis
};

template <typename T>
__device__ __forceinline__ T adj_pchip(T dl, T dr) {
  const T p = dl * dr;
  return p > T(0) ? (T(2) * p) / (dl + dr) : T(0);
}

template <typename T>
__device__ __forceinline__ T adj_slope(const T* u, int l, int stride, int g, int n) {
  if (g < 0 || g >= n) return T(0);
  const T* c = u + l * stride;
  if (g == 0) return adj_pchip(c[stride] - c[0], c[2 * stride] - c[stride]);
  if (g == n - 1) return adj_pchip(c[0] - c[-stride], c[-stride] - c[-2 * stride]);
  return adj_pchip(c[0] - c[-stride], c[stride] - c[0]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

template <typename T, int Q>
__global__ void __launch_bounds__(FK_THREADS) k_adj_scatter(const AdjArgs<T> g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Step2D<T>& a = g.s;
  const int lx = a.lx, ly = a.ly, lyr = a.lyr;
  V4<T>* R = reinterpret_cast<V4<T>*>(smem);
  V2<T>* S = reinterpret_cast<V2<T>*>(R + lx * lyr);
  T* U = reinterpret_cast<T*>(S + lx * lyr);
  T* DX = U + lx * ly;
  T* DY = DX + lx * ly;
  T* MU = DY + lx * ly;  // 3 lx ly accumulators, row-major like U
  __shared__ double red[4][FK_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = 1 + blockIdx.x * 32;
  const int k0 = 1 + blockIdx.y * a.ty;
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;
  const int64_t J = (int64_t)a.nx * a.ny;

  for (int lk = warp; lk < ly; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const bool rowin = gk >= 0 && gk < a.ny;
    for (int li = lane; li < lx; li += 32) {
      const int gi = gi0 + li;
      U[lk * lx + li] = (rowin && gi >= 0 && gi < a.nx) ? a.u_in[(int64_t)gk * a.nx + gi] : T(0);
      MU[lk * lx + li] = T(0);
      MU[lx * ly + lk * lx + li] = T(0);
      MU[2 * lx * ly + lk * lx + li] = T(0);
    }
  }
  __syncthreads();
  for (int lk = 1 + warp; lk <= ly - 2; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    const T* row = U + lk * lx;
    for (int li = 1 + lane; li <= lx - 2; li += 32) {
      DX[lk * lx + li] = adj_slope(row, li, 1, gi0 + li, a.nx);
      DY[lk * lx + li] = adj_slope(U + li, lk, lx, gk, a.ny);
    }
  }
  __syncthreads();
  for (int lk = 1 + warp; lk <= ly - 2; lk += FK_THREADS / 32) {
    for (int lc = 1 + lane; lc <= lx - 3; lc += 32) {
      const int o = lk * lx + lc;
      V4<T> r;
      r.x = U[o];
      r.y = U[o + 1] - U[o];
      r.z = DX[o];
      r.w = DX[o + 1];
      V2<T> s;
      s.x = DY[o];
      s.y = DY[o + 1] - DY[o];
      R[lc * lyr + lk] = r;
      S[lc * lyr + lk] = s;
    }
  }
  __syncthreads();

  double dth0 = 0.0, dth1 = 0.0, dth2 = 0.0, dth3 = 0.0;
  unsigned bad = 0;
  const int i = i0 + lane;
  const int li = i - gi0;
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (i > a.nx - 2 || k > a.ny - 2) continue;
    const T lam = g.lam[(int64_t)k * a.nx + i];
    if (lam == T(0)) continue;
    const int lk = k - gk0;
    T dx, dy, ax[3], ay[3];
    if (a.family == FK_CELLULAR_FLOW) {
      const T* ct = a.col_tab + 4 * (int64_t)i;
      const T* rt = a.row_tab + 2 * (int64_t)k;
      dx = a.kx * rt[0] * (a.A * ct[0] + a.e1 * ct[1]);
      dy = a.ky * rt[1] * (a.A * ct[2] + a.e2 * ct[3]);
      const T cx = a.kx * rt[0], cy = a.ky * rt[1];
      ax[0] = cx * ct[0];
      ay[0] = cy * ct[2];
      ax[1] = cx * g.st * ct[1];
      ay[1] = cy * T(2) * g.st * ct[3];
      ax[2] = cx * g.sw * ct[1];
      ay[2] = cy * T(2) * g.sw * ct[3];
    } else {
      dx = a.cdx;
      dy = a.cdy;
      ax[0] = g.cbx; ay[0] = T(0);
      ax[1] = T(0);  ay[1] = g.cby;
      ax[2] = T(0);  ay[2] = T(0);
    }
    // y factors: value and slope bases and their t-derivatives
    int rq[Q];
    T wy[Q], y00[Q], y01[Q], y10[Q], y11[Q], d01[Q], d10[Q], d11[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T d = dy + a.gy[q];
      const bool out = (d < T(-k)) || (d > T(a.ny - 1 - k));
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
      rq[q] = out ? lk : lc;
      wy[q] = out ? T(0) : a.w[q];
      const T t2 = t * t, omt = T(1) - t;
      y01[q] = t2 * (T(3) - T(2) * t);
      y00[q] = T(1) - y01[q];
      y10[q] = t * omt * omt;
      y11[q] = -(t2 * omt);
      d01[q] = T(6) * t * omt;                 // d h01 / dt (d h00/dt = -d01)
      d10[q] = omt * (T(1) - T(3) * t);        // d h10 / dt
      d11[q] = t * (T(3) * t - T(2));          // d h11 / dt
    }
    T Gx = T(0), Gy = T(0), Gxn = T(0), Gyn = T(0);
    for (int p = 0; p < Q; ++p) {
      const T d = dx + a.gx[p];
      if ((d < T(-i)) || (d > T(a.nx - 1 - i))) continue;
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
      const T x01 = t2 * (T(3) - T(2) * t), x00 = T(1) - x01;
      const T x10 = t * omt * omt, x11 = -(t2 * omt);
      const T e01 = T(6) * t * omt, e10 = omt * (T(1) - T(3) * t), e11 = t * (T(3) * t - T(2));
      const V4<T>* Rc = R + lc * lyr;
      const V2<T>* Sc = S + lc * lyr;
      const T wp = a.w[p], Wp = lam * wp;
      T gxp = T(0), gyp = T(0), gyn = T(0);
      for (int q = 0; q < Q; ++q) {
        if (wy[q] == T(0)) continue;
        const int r0i = rq[q];
        const V4<T> r0 = Rc[r0i];
        const V4<T> r1 = Rc[r0i + 1];
        const V2<T> s0 = Sc[r0i];
        const V2<T> s1 = Sc[r0i + 1];
        // interpolant along the two rows (value and x-derivative in t)
        const T v0 = r0.x + x01 * r0.y + x10 * r0.z + x11 * r0.w;
        const T v1 = r1.x + x01 * r1.y + x10 * r1.z + x11 * r1.w;
        const T dv0 = e01 * r0.y + e10 * r0.z + e11 * r0.w;
        const T dv1 = e01 * r1.y + e10 * r1.z + e11 * r1.w;
        const T b0 = s0.x + x01 * s0.y, b1 = s1.x + x01 * s1.y;
        const T db0 = e01 * s0.y, db1 = e01 * s1.y;
        const T wq = wy[q];
        const T dIx = y00[q] * dv0 + y01[q] * dv1 + y10[q] * db0 + y11[q] * db1;
        const T dIy = d01[q] * (v1 - v0) + d10[q] * b0 + d11[q] * b1;
        gxp += wq * dIx;
        gyp += wq * dIy;
        gyn += wq * dIy * a.gy[q];
        // transpose of the interpolation: 12 weights to the cell corners
        const T W = Wp * wq;
        const int o0 = (rq[q]) * lx + lc, o1 = o0 + lx;
        atomicAdd(&MU[o0], W * x00 * y00[q]);
        atomicAdd(&MU[o0 + 1], W * x01 * y00[q]);
        atomicAdd(&MU[o1], W * x00 * y01[q]);
        atomicAdd(&MU[o1 + 1], W * x01 * y01[q]);
        T* MX = MU + lx * ly;
        atomicAdd(&MX[o0], W * x10 * y00[q]);
        atomicAdd(&MX[o0 + 1], W * x11 * y00[q]);
        atomicAdd(&MX[o1], W * x10 * y01[q]);
        atomicAdd(&MX[o1 + 1], W * x11 * y01[q]);
        T* MY = MU + 2 * lx * ly;
        atomicAdd(&MY[o0], W * x00 * y10[q]);
        atomicAdd(&MY[o0 + 1], W * x01 * y10[q]);
        atomicAdd(&MY[o1], W * x00 * y11[q]);
        atomicAdd(&MY[o1 + 1], W * x01 * y11[q]);
      }
      Gx += wp * gxp;
      Gy += wp * gyp;
      Gxn += wp * gxp * a.gx[p];
      Gyn += wp * gyn;
    }
    const double l = (double)lam;
    dth0 += l * ((double)ax[0] * Gx + (double)ay[0] * Gy);
    dth1 += l * ((double)ax[1] * Gx + (double)ay[1] * Gy);
    dth2 += l * ((double)ax[2] * Gx + (double)ay[2] * Gy);
    dth3 += l * (double)g.cn * ((double)Gxn + (double)Gyn);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
  __syncthreads();
  // flush the tile's accumulators (halo included) into the global mu
  for (int lk = warp; lk < ly; lk += FK_THREADS / 32) {
    const int gk = gk0 + lk;
    if (gk < 0 || gk >= a.ny) continue;
    for (int li2 = lane; li2 < lx; li2 += 32) {
      const int gi = gi0 + li2;
      if (gi < 0 || gi >= a.nx) continue;
      const int64_t j = (int64_t)gk * a.nx + gi;
      const int o = lk * lx + li2;
      const T m0 = MU[o], m1 = MU[lx * ly + o], m2 = MU[2 * lx * ly + o];
      if (m0 != T(0)) atomicAdd(&g.mu[j], m0);
      if (m1 != T(0)) atomicAdd(&g.mu[J + j], m1);
      if (m2 != T(0)) atomicAdd(&g.mu[2 * J + j], m2);
    }
  }
  // FP64 reduction of the parameter derivatives
  dth0 = warp_sum(dth0);
  dth1 = warp_sum(dth1);
  dth2 = warp_sum(dth2);
  dth3 = warp_sum(dth3);
  if (lane == 0) {
    red[0][warp] = dth0;
    red[1][warp] = dth1;
    red[2][warp] = dth2;
    red[3][warp] = dth3;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < FK_THREADS / 32; ++w) s += red[threadIdx.x][w];
    if (s != 0.0) atomicAdd(&g.dth[threadIdx.x], s);
  }
}

// ------------------------------------------- masked tensor-window adjoint
// For an FP32 plan eligible for the masked step kernel the forward step is
// u^n_j = u_j + sum_{c,r} [(u_{c,r} - u_j) phi_c Phi_r + X_{c,r} psi_c Phi_r
//                          + Y_{c,r} phi_c Psi_r] + (1 - u_j) E
// over the node's W x W window (X, Y the scaled slopes; phi, psi and Phi,
// Psi the x and y Hermite weights of the node's points, exiting points
// dropped; E the exit mass).  Its transpose is rank one per node:
//   mu_u += lambda phi_c Phi_r,  mu_X += lambda psi_c Phi_r,  mu_Y += lambda phi_c Psi_r
// (the explicit u_j terms cancel: the in-box weights and E sum to one).
// The parameter derivatives need the weights' derivatives in the point
// positions: phi^d = sum_p w_p V'(.), the same for psi, and phi^g with each
// point scaled by its offset g_p (the sigma direction); Gx = sum (u - u_j)
// phi^d Phi + X psi^d Phi + Y phi^d Psi, and Gy, Gxn, Gyn alike.  Each
// of these is a double sum of one rank-one weight against the window, so
// one pass suffices: it scatters mu and forms the row sums (contracted
// with the y derivatives: Gy, Gyn) and the column sums (contracted with
// the x derivatives: Gx, Gxn).

// Weighted cubic Hermite node functions of one point at local position t
// in its cell: values (v0, v1), slopes (s0, s1), and their t-derivatives.
struct HermW {
  float v0, v1, s0, s1, dv0, dv1, ds0, ds1;
};
__device__ __forceinline__ HermW herm_w(float w, float t) {
  HermW h;
  const float tt = t * t, omt = 1.f - t;
  h.v1 = w * (tt * (3.f - 2.f * t));
  h.v0 = w - h.v1;
  h.s0 = w * (t * omt * omt);
  h.s1 = -w * (tt * omt);
  h.dv1 = w * (6.f * t * omt);
  h.dv0 = -h.dv1;
  h.ds0 = w * (omt * (1.f - 3.f * t));
  h.ds1 = w * (t * (3.f * t - 2.f));
  return h;
}

// A set of K weight arrays over W window slots, and the uniform scatter of
// one point's (a, b) node pair into slots (m + beta, m + beta + 1).
template <int W, int K>
struct Slots {
  float v[K][W];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int s = 0; s < W; ++s) v[k][s] = 0.f;
  }
};
template <int W, int K, int M>
struct SlotAdd {
  __device__ __forceinline__ static void run(int m, bool beta, Slots<W, K>& S, const float (&a)[K],
                                             const float (&b)[K]) {
    if (m == M) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        S.v[k][M] += beta ? 0.f : a[k];
        S.v[k][M + 1] += beta ? a[k] : b[k];
        S.v[k][M + 2] += beta ? b[k] : 0.f;
      }
    } else {
      SlotAdd<W, K, M + 1>::run(m, beta, S, a, b);
    }
  }
};
template <int W, int K>
struct SlotAdd<W, K, W - 2> {
  __device__ __forceinline__ static void run(int, bool, Slots<W, K>&, const float (&)[K],
                                             const float (&)[K]) {}
};

// 1D weights of one axis over the window slots, point position z + g_q
// after the window origin, exiting points (outside [lo, hi]) dropped.
// K = 2: values and slopes; K = 4: their position derivatives, plain and
// times the point's offset g_q.
template <int Q, int W, int K>
__device__ __forceinline__ void axis_weights(Slots<W, K>& S, const Step2D<float>& a, float z,
                                             const float* gq_all, float lo, float hi) {
  S.zero();
#pragma unroll 1
  for (int q = 0; q < Q; ++q) {
    const float sq = z + gq_all[q], tp = sq - a.wmf[q];
    const bool beta = tp >= 1.f;
    const float w = (sq < lo || sq > hi) ? 0.f : a.w[q];
    const HermW h = herm_w(w, beta ? tp - 1.f : tp);
    if constexpr (K == 2) {
      const float A[2] = {h.v0, h.s0}, B[2] = {h.v1, h.s1};
      SlotAdd<W, 2, 0>::run(a.wm[q], beta, S, A, B);
    } else {
      const float gq = gq_all[q];
      const float A[4] = {h.dv0, h.ds0, h.dv0 * gq, h.ds0 * gq};
      const float B[4] = {h.dv1, h.ds1, h.dv1 * gq, h.ds1 * gq};
      SlotAdd<W, 4, 0>::run(a.wm[q], beta, S, A, B);
    }
  }
}

// Weight tables (adj_tables): float4 quadruples [axis][slot][quad][piece]
// after kTabHead float4 of piece starts [axis][piece]; quad 0 {V3, S3, V2,
// S2} and 1 {V1, S1, V0, S0}, the value/slope cubics in u = zeta - start;
// quad 2 {G2v, G2s, G1v, G1s} and 3 {G0v, G0s, 0, 0}, the quadratics of
// the position derivatives times the point offsets.
constexpr int kTabHead = 2 * FK_MAXQ_2D / 4;
__host__ __device__ constexpr int adj_tab_float4(int W) { return kTabHead + 2 * W * 4 * FK_MAXQ_2D; }

__device__ __forceinline__ int adj_piece(const float* brk, int nb, float zeta) {
  int k = 0;
  for (int b = 0; b < nb; ++b) k += zeta >= brk[b] ? 1 : 0;
  return k;
}

// values and slopes (K = 2), or position derivatives plain and times the
// point offsets (K = 4), of one axis from its table
template <int W, int K>
__device__ __forceinline__ void tab_weights(Slots<W, K>& S, const float4* TB, int axis, int piece,
                                            float u) {
  const float2 U = f2(u, u);
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const float4* e = TB + kTabHead + ((axis * W + c) * 4) * FK_MAXQ_2D + piece;
    const float4 h = e[0], l = e[FK_MAXQ_2D];
    if constexpr (K == 2) {
      const float2 v = fma2(fma2(fma2(f2(h.x, h.y), U, f2(h.z, h.w)), U, f2(l.x, l.y)), U,
                            f2(l.z, l.w));
      S.v[0][c] = v.x;
      S.v[1][c] = v.y;
    } else {
      // d/du of the cubic: (3 c3 u + 2 c2) u + c1
      const float2 d = fma2(fma2(mul2(f2(3.f, 3.f), f2(h.x, h.y)), U, mul2(f2(2.f, 2.f), f2(h.z, h.w))),
                            U, f2(l.x, l.y));
      const float4 q2 = e[2 * FK_MAXQ_2D], q0 = e[3 * FK_MAXQ_2D];
      const float2 gq = fma2(fma2(f2(q2.x, q2.y), U, f2(q2.z, q2.w)), U, f2(q0.x, q0.y));
      S.v[0][c] = d.x;
      S.v[1][c] = d.y;
      S.v[2][c] = gq.x;
      S.v[3][c] = gq.y;
    }
  }
}

// Drift of node (i, k) over one step in cells (dt b / h), the same
// expression as the forward step's.
__device__ __forceinline__ void node_drift(const Step2D<float>& a, int i, int k, float& dx,
                                           float& dy) {
  if (a.family == FK_CELLULAR_FLOW) {
    const float* ct = a.col_tab + 4 * (int64_t)i;
    const float* rt = a.row_tab + 2 * (int64_t)k;
    dx = a.kx * rt[0] * (a.A * ct[0] + a.e1 * ct[1]);
    dy = a.ky * rt[1] * (a.A * ct[2] + a.e2 * ct[3]);
  } else {
    dx = a.cdx;
    dy = a.cdy;
  }
}

// Position of a node's points along one axis, in cells after the window
// origin (the cell of point 0): z = offset of point 0, [lo, hi] the box;
// whether all points stay inside, and then point 0's table piece and its
// offset u in it.
struct AxisPos {
  float z, lo, hi, u;
  int piece;
  bool inside;
};
template <int Q>
__device__ __forceinline__ AxisPos axis_pos(float d, float g0, int node, int n, const float* brk,
                                            float last, const float4* TB, int axis) {
  AxisPos P;
  const float f0 = floorf(d + g0);
  P.z = d - f0;
  P.lo = -(float)node - f0;
  P.hi = (float)(n - 1 - node) - f0;
  const float e = (d + g0) - f0;
  P.inside = e >= P.lo && e + last <= P.hi;
  P.piece = adj_piece(brk, Q - 1, e);
  P.u = e - reinterpret_cast<const float*>(TB)[axis * FK_MAXQ_2D + P.piece];
  return P;
}

// Gradient of the slope rule H(dl, dr) = 2 dl dr / (dl + dr) (dl dr > 0,
// else 0) of Eq. (e300): dH/d dl = 2 (dr / (dl + dr))^2 and
// dH/d dr = 2 (dl / (dl + dr))^2, 0 on the zero branch.  Formed from the
// ratios, which lie in [0, 1]: differences near the bottom of the exponent
// range (a march from the indicator leaves such values far from the
// boundary) would overflow 1 / (dl + dr)^2.
template <typename T>
__device__ __forceinline__ void harm_grad(T dl, T dr, T& gl, T& gr) {
  if (dl * dr > T(0)) {
    const T ql = dl / (dl + dr), qr = T(1) - ql;  // dr / (dl + dr)
    gl = T(2) * qr * qr;
    gr = T(2) * ql * ql;
  } else {
    gl = T(0);
    gr = T(0);
  }
}

// Transposed slope map along one grid line, at node i of n (u and mu point
// at node i, s is the stride between neighbours): the sum over the slopes
// m = i-1, i, i+1 that read u_i of mu_m dH_m/du_i, where slope m reads
// dl = u_m - u_{m-1} and dr = u_{m+1} - u_m.  The end rule stated after
// Eq. (e300) makes the slope of node 0 the same function of u as that of
// node 1 (the harmonic mean is symmetric), and node n-1 that of node n-2,
// so mu of the end nodes is added to their neighbours' and only interior
// three-point slopes remain.
// Every load is made, at an offset clamped into the line, before any term
// is chosen: the ten loads are then in flight together instead of each
// waiting behind the range test that guards it (a clamped load reads a
// real node, and the terms it feeds are dropped by the same tests as
// before, in the same order).
template <typename T>
__device__ __forceinline__ T slope_line_t(const T* u, const T* mu, int64_t s, int n, int i) {
  auto off = [&](int d) { return (int64_t)(min(max(i + d, 0), n - 1) - i) * s; };
  const T um2 = u[off(-2)], um1 = u[off(-1)], u0 = u[0], up1 = u[off(1)], up2 = u[off(2)];
  const T mm2 = mu[off(-2)], mm1 = mu[off(-1)], m0 = mu[0], mp1 = mu[off(1)], mp2 = mu[off(2)];
  // mu of slope m = i + d (mc), end nodes folded in (mlo: node m - 1, mhi: node m + 1)
  auto mu_f = [&](int d, T mlo, T mc, T mhi) {
    const int m = i + d;
    T v = mc;
    if (m == 1) v += mlo;
    if (m == n - 2) v += mhi;
    return (m < 1 || m > n - 2) ? T(0) : v;
  };
  T acc = T(0), gl, gr;
  harm_grad(um1 - um2, u0 - um1, gl, gr);  // slope i-1: u_i is its right node
  if (i >= 2) acc += mu_f(-1, mm2, mm1, m0) * gr;
  harm_grad(u0 - um1, up1 - u0, gl, gr);  // slope i
  if (i >= 1 && i <= n - 2) acc += mu_f(0, mm1, m0, mp1) * (gl - gr);
  harm_grad(up1 - u0, up2 - up1, gl, gr);  // slope i+1: u_i is its left node
  if (i <= n - 3) acc -= mu_f(1, m0, mp1, mp2) * gl;
  return acc;
}

// Rows of a masked-adjoint tile whose lambda the kernel can form itself
// (its tile height may not exceed this when lam == nullptr).
constexpr int kAdjLamRows = 16;

// lambda^n at interior node (i, k): read, or (lam == nullptr) the slope
// transpose of the previous step's accumulators, as k_adj_slopes_t forms
// it, after which the node's accumulators of the step after this one (and
// those of the boundary nodes next to it, which no tile owns) are zeroed.
__device__ __forceinline__ float node_lambda(const AdjArgs<float>& g, int i, int k) {
  const int nx = g.s.nx, ny = g.s.ny;
  const int64_t J = (int64_t)nx * ny, j = (int64_t)k * nx + i;
  if (g.lam) return g.lam[j];
  const float* mu = g.mu_prev;
  const float lam = mu[j] + slope_line_t(g.u_prev + j, mu + J + j, (int64_t)1, nx, i) +
                    slope_line_t(g.u_prev + j, mu + 2 * J + j, (int64_t)nx, ny, k);
  auto clear = [&](int64_t m) {
    g.mu_clear[m] = 0.f;
    g.mu_clear[J + m] = 0.f;
    g.mu_clear[2 * J + m] = 0.f;
  };
  clear(j);
  const bool L = i == 1, R = i == nx - 2, B = k == 1, T = k == ny - 2;
  if (L) clear(j - 1);
  if (R) clear(j + 1);
  if (B) clear(j - nx);
  if (T) clear(j + nx);
  if (L && B) clear(j - nx - 1);
  if (R && B) clear(j - nx + 1);
  if (L && T) clear(j + nx - 1);
  if (R && T) clear(j + nx + 1);
  return lam;
}

// Register budget for kAdjMinBlocks CTAs per SM (80 registers): the window
// pass keeps only the 1D weights and the column sums in registers.
#ifndef FK_ADJ_MINB
#define FK_ADJ_MINB 3
#endif
constexpr int kAdjMinBlocks = FK_ADJ_MINB;
template <int Q, int W>
__global__ void __launch_bounds__(FK_THREADS, kAdjMinBlocks) k_adj_masked(const AdjArgs<float> g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Step2D<float>& a = g.s;
  const int lx = a.lx, ly = a.ly, lp = a.lyr;
  float4* TB = reinterpret_cast<float4*>(smem);  // weight tables
  float4* Rec = TB + adj_tab_float4(W);
  float* U = reinterpret_cast<float*>(Rec + ly * lp);
  // the tile's mu accumulators: 3 planes of ly x lp (mu_u, mu_X, mu_Y) in
  // fixed point, because 32-bit integer adds are the shared-memory atomics
  // the hardware has (a float add is a compare-and-swap loop)
  int* MU = reinterpret_cast<int*>(U + ly * lp);
  float* RS = reinterpret_cast<float*>(MU + 3 * ly * lp);  // per-thread row sums A_r, B_r
  __shared__ float lred[FK_THREADS / 32];
  __shared__ int fred[4][FK_THREADS / 32];
  __shared__ float lam_s[kAdjLamRows][32];  // lambda^n of the thread's nodes (lam == nullptr)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = 1 + blockIdx.x * 32, k0 = 1 + blockIdx.y * a.ty;
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;
  const int i = i0 + lane, li = i - gi0;
  for (int e = tid; e < 3 * ly * lp; e += FK_THREADS) MU[e] = 0;
  for (int e = tid; e < adj_tab_float4(W); e += FK_THREADS) TB[e] = g.tab[e];
  {
    // Fixed-point scale S (a power of two).  A node's 1D value weights are
    // non-negative and sum to at most 1, its slope weights are at most 4/27
    // in absolute value, so each of its contributions to a cell is at most
    // |lambda_j|.  A cell is in the window of node j only if the window
    // origin i_j + floor(dx_j + g_0) lies in the W columns up to the cell,
    // so at most W + (spread of those floors over the tile) node columns,
    // and as many rows, reach it: every accumulator stays below
    // max|lambda| (W + spread_x)(W + spread_y), which S puts below 2^30.
    float lmax = 0.f;
    int fxl = INT_MAX, fxh = INT_MIN, fyl = INT_MAX, fyh = INT_MIN;
    for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
      const int k = k0 + ty;
      if (i > a.nx - 2 || k > a.ny - 2) break;
      const float lam = node_lambda(g, i, k);
      if (!g.lam) lam_s[ty][lane] = lam;
      if (lam == 0.f) continue;
      float dx, dy;
      node_drift(a, i, k, dx, dy);
      const int fx = (int)floorf(dx + a.gx[0]), fy = (int)floorf(dy + a.gy[0]);
      lmax = fmaxf(lmax, fabsf(lam));
      fxl = min(fxl, fx);
      fxh = max(fxh, fx);
      fyl = min(fyl, fy);
      fyh = max(fyh, fy);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, m));
      fxl = min(fxl, __shfl_xor_sync(0xffffffffu, fxl, m));
      fxh = max(fxh, __shfl_xor_sync(0xffffffffu, fxh, m));
      fyl = min(fyl, __shfl_xor_sync(0xffffffffu, fyl, m));
      fyh = max(fyh, __shfl_xor_sync(0xffffffffu, fyh, m));
    }
    if (lane == 0) {
      lred[warp] = lmax;
      fred[0][warp] = fxl;
      fred[1][warp] = fxh;
      fred[2][warp] = fyl;
      fred[3][warp] = fyh;
    }
  }
  masked_stage(a, Rec, U, gi0, gk0);  // ends with a barrier
  int s_exp = 0;  // S = 2^s_exp
  {
    float lmax = 0.f;
    int fxl = INT_MAX, fxh = INT_MIN, fyl = INT_MAX, fyh = INT_MIN;
#pragma unroll
    for (int w = 0; w < FK_THREADS / 32; ++w) {
      lmax = fmaxf(lmax, lred[w]);
      fxl = min(fxl, fred[0][w]);
      fxh = max(fxh, fred[1][w]);
      fyl = min(fyl, fred[2][w]);
      fyh = max(fyh, fred[3][w]);
    }
    if (lmax > 0.f) {
      const float ncov = (float)(W + fxh - fxl) * (float)(W + fyh - fyl);
      int b_exp = 0;
      frexpf(lmax * ncov, &b_exp);  // bound < 2^b_exp
      s_exp = min(30 - b_exp, 126);
    }
  }

  // per-thread sums of the parameter derivatives over the thread's few
  // nodes (in shared memory: registers go to the window pass); the sums
  // over the tile and the grid are FP64
  float* DA = RS + 2 * W * FK_THREADS + tid;
#pragma unroll
  for (int m = 0; m < 4; ++m) DA[m * FK_THREADS] = 0.f;
  unsigned bad = 0;
  int* MX = MU + ly * lp;
  int* MY = MX + ly * lp;
#pragma unroll 1
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (i > a.nx - 2 || k > a.ny - 2) break;
    const float lam = g.lam ? g.lam[(int64_t)k * a.nx + i] : lam_s[ty][lane];
    const float lamS = ldexpf(lam, s_exp);  // scaled to the accumulators' fixed point
    if (lamS == 0.f) continue;
    const int lk = k - gk0;
    const float uj = U[lk * lp + li];
    float dx, dy;
    node_drift(a, i, k, dx, dy);
    const float fx0 = floorf(dx + a.gx[0]), fy0 = floorf(dy + a.gy[0]);
    int wx = li + (int)fx0, wy = lk + (int)fy0;
    if (wx < 1 || wx + W - 1 > lx - 2 || wy < 1 || wy + W - 1 > ly - 2) {
      bad = 1u;
      wx = 1;
      wy = 1;
    }
    Slots<W, 2> YV, XV;  // (Phi, Psi) and (phi, psi)
    {
      const AxisPos X = axis_pos<Q>(dx, a.gx[0], i, a.nx, g.brk[0], g.last[0], TB, 0);
      const AxisPos Y = axis_pos<Q>(dy, a.gy[0], k, a.ny, g.brk[1], g.last[1], TB, 1);
      if (X.inside && Y.inside) {
        tab_weights(YV, TB, 1, Y.piece, Y.u);
        tab_weights(XV, TB, 0, X.piece, X.u);
      } else {
        axis_weights<Q>(YV, a, Y.z, a.gy, Y.lo, Y.hi);
        axis_weights<Q>(XV, a, X.z, a.gx, X.lo, X.hi);
      }
    }
    // one pass over the window: the transposed scatter, the row sums
    //   A_r = sum_c (u - u_j) phi_c + X psi_c,  B_r = sum_c Y phi_c
    // and the column sums
    //   C_c = sum_r (u - u_j) Phi_r + Y Psi_r,  D_c = sum_r X Phi_r
    // (the y and x position derivatives then contract with the row and
    // the column sums respectively)
    // (A_r, B_r kept in shared memory, thread-minor: registers go to the
    // window pass)
    float* AR = RS + tid;
    float* BR = RS + W * FK_THREADS + tid;
    float2 CD[W];  // (C_c, D_c)
#pragma unroll
    for (int c = 0; c < W; ++c) CD[c] = f2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const int o = (wy + r) * lp + wx;
      const float4* row = Rec + o;
      const float Pr = YV.v[0][r], Sr = YV.v[1][r];
      const float lP = lamS * Pr, lS = lamS * Sr;
      const float2 PP = f2(Pr, Pr), LP = f2(lP, lP);
      float2 AE = f2(0.f, 0.f);
      float Br = 0.f;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float4 v = row[c];
        const float2 ex = f2(v.x - uj, v.y);
        const float2 ph = f2(XV.v[0][c], XV.v[1][c]);
        AE = fma2(ph, ex, AE);
        Br = fmaf(ph.x, v.z, Br);
        CD[c] = fma2(PP, ex, CD[c]);
        CD[c].x = fmaf(Sr, v.z, CD[c].x);
        const float2 m = mul2(LP, ph);
        atomicAdd(&MU[o + c], __float2int_rn(m.x));
        atomicAdd(&MX[o + c], __float2int_rn(m.y));
        atomicAdd(&MY[o + c], __float2int_rn(lS * ph.x));
      }
      AR[r * FK_THREADS] = AE.x + AE.y;
      BR[r * FK_THREADS] = Br;
    }
    // the positions again, recomputed from the drift rather than held
    // through the window pass
    const AxisPos X = axis_pos<Q>(opaque(dx), a.gx[0], i, a.nx, g.brk[0], g.last[0], TB, 0);
    const AxisPos Y = axis_pos<Q>(opaque(dy), a.gy[0], k, a.ny, g.brk[1], g.last[1], TB, 1);
    const bool inside = X.inside && Y.inside;
    float Gy = 0.f, Gyn = 0.f, Gx = 0.f, Gxn = 0.f;
    {
      Slots<W, 4> YD;  // y position derivatives, plain and times g_q
      if (inside)
        tab_weights(YD, TB, 1, Y.piece, Y.u);
      else
        axis_weights<Q>(YD, a, Y.z, a.gy, Y.lo, Y.hi);
#pragma unroll
      for (int r = 0; r < W; ++r) {
        const float Ar = AR[r * FK_THREADS], Br = BR[r * FK_THREADS];
        Gy = fmaf(YD.v[0][r], Ar, fmaf(YD.v[1][r], Br, Gy));
        Gyn = fmaf(YD.v[2][r], Ar, fmaf(YD.v[3][r], Br, Gyn));
      }
    }
    {
      Slots<W, 4> XD;  // x position derivatives, plain and times g_p
      if (inside)
        tab_weights(XD, TB, 0, X.piece, X.u);
      else
        axis_weights<Q>(XD, a, X.z, a.gx, X.lo, X.hi);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        Gx = fmaf(XD.v[0][c], CD[c].x, fmaf(XD.v[1][c], CD[c].y, Gx));
        Gxn = fmaf(XD.v[2][c], CD[c].x, fmaf(XD.v[3][c], CD[c].y, Gxn));
      }
    }
    // d(shift in cells)/d theta per axis (the derivative of the drift in
    // A, eps, omega; or in b_1, b_2)
    float ax[3], ay[3];
    if (a.family == FK_CELLULAR_FLOW) {
      const float* ct = a.col_tab + 4 * (int64_t)i;
      const float* rt = a.row_tab + 2 * (int64_t)k;
      const float cx = a.kx * rt[0], cy = a.ky * rt[1];
      ax[0] = cx * ct[0];
      ay[0] = cy * ct[2];
      ax[1] = cx * g.st * ct[1];
      ay[1] = cy * 2.f * g.st * ct[3];
      ax[2] = cx * g.sw * ct[1];
      ay[2] = cy * 2.f * g.sw * ct[3];
    } else {
      ax[0] = g.cbx; ay[0] = 0.f;
      ax[1] = 0.f;   ay[1] = g.cby;
      ax[2] = 0.f;   ay[2] = 0.f;
    }
    DA[0] += lam * (ax[0] * Gx + ay[0] * Gy);
    DA[FK_THREADS] += lam * (ax[1] * Gx + ay[1] * Gy);
    DA[2 * FK_THREADS] += lam * (ax[2] * Gx + ay[2] * Gy);
    DA[3 * FK_THREADS] += lam * g.cn * (Gxn + Gyn);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
  __syncthreads();
  // flush the tile's accumulators (halo included) into the global mu
  const int64_t J = (int64_t)a.nx * a.ny;
  const float fix_inv = ldexpf(1.f, -s_exp);
  for (int r = warp; r < ly; r += FK_THREADS / 32) {
    const int gk = gk0 + r;
    if (gk < 0 || gk >= a.ny) continue;
    for (int c = lane; c < lx; c += 32) {
      const int gi = gi0 + c;
      if (gi < 0 || gi >= a.nx) continue;
      const int64_t j = (int64_t)gk * a.nx + gi;
      const int o = r * lp + c;
      const float m0 = (float)MU[o] * fix_inv, m1 = (float)MX[o] * fix_inv,
                  m2 = (float)MY[o] * fix_inv;
      if (m0 != 0.f) atomicAdd(&g.mu[j], m0);
      if (m1 != 0.f) atomicAdd(&g.mu[J + j], m1);
      if (m2 != 0.f) atomicAdd(&g.mu[2 * J + j], m2);
    }
  }
  // tile sums of the parameter derivatives (the per-thread sums are visible
  // since the barrier above): warp q < 4 adds up quantity q, 8 per-thread
  // sums per lane in FP32, then the lanes in FP64 (the FP64 pipe is slow:
  // one reduction per quantity, not one per warp)
  if (warp < 4) {
    const float* dq = RS + 2 * W * FK_THREADS + warp * FK_THREADS;
    float part = 0.f;
#pragma unroll
    for (int m = 0; m < FK_THREADS / 32; ++m) part += dq[lane + 32 * m];
    const double sum = warp_sum((double)part);
    if (lane == 0 && sum != 0.0) atomicAdd(&g.dth[warp], sum);
  }
}

// lambda^{n+1}_i = mu_u[i] + sum_m mu_x[m] dD^x_m/du_i + sum_m mu_y[m] dD^y_m/du_i;
// also clears node i of the other mu buffer, which the next backward step
// accumulates into
template <typename T>
__global__ void k_adj_slopes_t(const T* __restrict__ u, const T* __restrict__ mu,
                               T* __restrict__ lam_out, T* __restrict__ mu_next, int nx,
                               int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || k >= ny) return;
  const int64_t J = (int64_t)nx * ny, j = (int64_t)k * nx + i;
  lam_out[j] = mu[j] + slope_line_t(u + j, mu + J + j, (int64_t)1, nx, i) +
               slope_line_t(u + j, mu + 2 * J + j, (int64_t)nx, ny, k);
  mu_next[j] = T(0);
  mu_next[J + j] = T(0);
  mu_next[2 * J + j] = T(0);
}

template <typename T>
__global__ void k_cast_in(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = (T)src[j];
}

// dynamic shared memory of the scatter kernel (+ 256 B of static reduction space)
size_t adj_smem(int lx, int ly, int lyr, int elem) {
  return fk_step2d_smem(lx, ly, lyr, elem) + (size_t)3 * lx * ly * elem;
}
const size_t kAdjStatic = 4 * (FK_THREADS / 32) * sizeof(double);

template <typename T, int Q>
cudaError_t launch_adj_q(const AdjArgs<T>& g, cudaStream_t s) {
  const size_t smem = adj_smem(g.s.lx, g.s.ly, g.s.lyr, (int)sizeof(T));
  static bool set = false;
  if (!set) {
    // dynamic + static shared memory must stay within the opt-in limit
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_adj_scatter<T, Q>);
    int dev = 0, optin = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_adj_scatter<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    set = true;
  }
  dim3 grid((g.s.nx - 2 + 31) / 32, (g.s.ny - 2 + g.s.ty - 1) / g.s.ty);
  k_adj_scatter<T, Q><<<grid, FK_THREADS, smem, s>>>(g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj(const AdjArgs<T>& g, int q, cudaStream_t s) {
  switch (q) {
#define FK_CASE(QQ) \
  case QQ: return launch_adj_q<T, QQ>(g, s);
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

size_t adj_masked_smem(int ly, int lp, int w) {
  return (size_t)adj_tab_float4(w) * 16 + (size_t)ly * lp * (16 + 4 + 12) +
         (size_t)2 * w * FK_THREADS * 4 + (size_t)4 * FK_THREADS * 4;
}

// The piecewise-cubic weight tables of the masked adjoint, per axis.  With
// point 0 at fractional cell position zeta in [0, 1) after the window
// origin, point q sits at zeta + D_q (D_q = g_q - g_0).  The value weight of
// window slot s is phi_s(zeta) = sum_q w_q V(zeta + D_q - s), the slope
// weight psi_s the same with S; V, S are the cubic Hermite node functions
// (h00, h01, h10, h11 of Eq. (Lag11) in one piece each).  Both are cubic in
// zeta between the positions where some point crosses a cell boundary,
// zeta = 1 - frac(D_q): at most Q pieces.  d phi_s / d zeta is the weight
// of the common position derivative (the drift direction); the sigma
// direction needs sum_q w_q g_q V'(...), a quadratic per piece.  All are
// expanded in u = zeta - (start of the piece, as float).  The weights are
// continuous in zeta (the node functions are C^1), so a zeta that rounds
// across a piece boundary takes either piece.
bool adj_tables(fk_plan* p, std::vector<float>& tab) {
  const int Q = p->q, W = p->mwin;
  const size_t head = 4 * kTabHead;
  tab.assign((size_t)4 * adj_tab_float4(W), 0.f);
  const double sg = (p->coeffs.family == FK_CONST_DRIFT ? p->coeffs.p[3] : sqrt(2.0 * p->coeffs.p[3])) *
                    sqrt(2.0 * p->dt);
  for (int m = 0; m < 2; ++m) {
    double gq[FK_MAXQ_2D];
    for (int q = 0; q < Q; ++q) gq[q] = (double)(float)(sg * p->gh_a[q] / p->h[m]);
    std::vector<double> br;
    for (int q = 1; q < Q; ++q) {
      const double d = gq[q] - gq[0], f = d - floor(d);
      if (f > 0.0) br.push_back((double)(float)(1.0 - f));
    }
    std::sort(br.begin(), br.end());
    br.erase(std::unique(br.begin(), br.end()), br.end());
    const int P = (int)br.size() + 1;
    if (P > FK_MAXQ_2D) return false;
    for (int b = 0; b < FK_MAXQ_2D; ++b) p->adj_break[m][b] = b < P - 1 ? (float)br[b] : 2.0f;
    p->adj_last[m] = (float)(gq[Q - 1] - gq[0]);
    for (int k = 0; k < P; ++k) {
      const double a0 = k == 0 ? 0.0 : br[k - 1], a1 = k == P - 1 ? 1.0 : br[k];
      const double mid = 0.5 * (a0 + a1);
      double V[FK_MAXQ_2D + 8][4] = {}, S[FK_MAXQ_2D + 8][4] = {};
      double GV[FK_MAXQ_2D + 8][3] = {}, GS[FK_MAXQ_2D + 8][3] = {};
      for (int q = 0; q < Q; ++q) {
        const double D = gq[q] - gq[0];
        const int o = (int)floor(mid + D);  // cell of point q over this piece
        if (o < 0 || o + 1 > W - 1) return false;
        const double t0 = a0 + D - o;      // its local coordinate at u = 0
        // t = t0 + u: coefficients of t, t^2, t^3 in powers of u
        const double c1[4] = {t0, 1.0, 0.0, 0.0};
        const double c2[4] = {t0 * t0, 2.0 * t0, 1.0, 0.0};
        const double c3[4] = {t0 * t0 * t0, 3.0 * t0 * t0, 3.0 * t0, 1.0};
        const double w = p->gh_w[q], wg = w * gq[q];
        for (int e = 0; e < 4; ++e) {
          const double h01 = 3.0 * c2[e] - 2.0 * c3[e];
          const double h00 = (e == 0 ? 1.0 : 0.0) - h01;
          const double h10 = c1[e] - 2.0 * c2[e] + c3[e];
          const double h11 = c3[e] - c2[e];
          V[o][e] += w * h00;
          V[o + 1][e] += w * h01;
          S[o][e] += w * h10;
          S[o + 1][e] += w * h11;
        }
        for (int e = 0; e < 3; ++e) {  // d/du of the same cubics, times g_q
          const double d01 = (e + 1) * (3.0 * c2[e + 1] - 2.0 * c3[e + 1]);
          const double d10 = (e + 1) * (c1[e + 1] - 2.0 * c2[e + 1] + c3[e + 1]);
          const double d11 = (e + 1) * (c3[e + 1] - c2[e + 1]);
          GV[o][e] -= wg * d01;
          GV[o + 1][e] += wg * d01;
          GS[o][e] += wg * d10;
          GS[o + 1][e] += wg * d11;
        }
      }
      tab[m * FK_MAXQ_2D + k] = (float)a0;
      for (int c = 0; c < W; ++c) {
        auto quad = [&](int j) { return &tab[head + 4 * ((size_t)((m * W + c) * 4 + j) * FK_MAXQ_2D + k)]; };
        float* q0 = quad(0);
        q0[0] = (float)V[c][3]; q0[1] = (float)S[c][3]; q0[2] = (float)V[c][2]; q0[3] = (float)S[c][2];
        float* q1 = quad(1);
        q1[0] = (float)V[c][1]; q1[1] = (float)S[c][1]; q1[2] = (float)V[c][0]; q1[3] = (float)S[c][0];
        float* q2 = quad(2);
        q2[0] = (float)GV[c][2]; q2[1] = (float)GS[c][2]; q2[2] = (float)GV[c][1]; q2[3] = (float)GS[c][1];
        float* q3 = quad(3);
        q3[0] = (float)GV[c][0]; q3[1] = (float)GS[c][0];
      }
    }
  }
  return true;
}

template <int Q, int W>
cudaError_t launch_adj_masked_qw(const AdjArgs<float>& g, cudaStream_t s) {
  const size_t smem = adj_masked_smem(g.s.ly, g.s.lyr, W);
  static bool set = false;
  if (!set) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_adj_masked<Q, W>);
    int dev = 0, optin = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_adj_masked<Q, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    set = true;
  }
  dim3 grid((g.s.nx - 2 + 31) / 32, (g.s.ny - 2 + g.s.ty - 1) / g.s.ty);
  k_adj_masked<Q, W><<<grid, FK_THREADS, smem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_adj_masked(const AdjArgs<float>& g, int q, cudaStream_t s) {
#define FK_M(QQ, WW) \
  if (q == QQ && g.s.win == WW) return launch_adj_masked_qw<QQ, WW>(g, s);
  FK_MASKED_LIST(FK_M)
#undef FK_M
  return cudaErrorInvalidValue;
}

// Whether the backward steps of plan p use the masked window form (FP32
// plans eligible for the masked step kernel; FK_ADJ_KERNEL=scatter|masked
// chooses explicitly where both apply), and its tile height.
bool adj_masked_built(int q, int w) {
#define FK_M(QQ, WW) \
  if (q == QQ && w == WW) return true;
  FK_MASKED_LIST(FK_M)
#undef FK_M
  return false;
}
bool adj_use_masked(const fk_plan* p) {
  if (p->prec != FK_FP32 || p->mwin <= 0 || !adj_masked_built(p->q, p->mwin)) return false;
  const char* k = getenv("FK_ADJ_KERNEL");
  return !(k && strcmp(k, "scatter") == 0);
}
int adj_masked_ty(const fk_plan* p, int smem_max) {
  const int lx = 32 + 2 * p->mhalo[0] + 2;
  auto bytes = [&](int ty) {  // (+ the kernel's static arrays: reductions and lam_s)
    return adj_masked_smem(ty + 2 * p->mhalo[1] + 2, lx | 1, p->mwin) + kAdjStatic +
           sizeof(float) * kAdjLamRows * 32;
  };
  // FK_ADJ_TILE=ty: an explicit tile height (profiling)
  if (const char* t = getenv("FK_ADJ_TILE")) {
    const int ty = atoi(t);
    if (ty >= 4 && ty <= 32 && bytes(ty) <= (size_t)smem_max) return ty;
  }
  // the tallest tile (<= 16 rows) with which kAdjMinBlocks CTAs share an
  // SM, else the tallest that fits at all
  int sm_smem = 0;
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
  for (int ty = 16; ty >= 4; ty -= 4)
    if (kAdjMinBlocks * (bytes(ty) + 1024) <= (size_t)sm_smem) return ty;
  for (int ty = 16; ty >= 4; ty -= 4)
    if (bytes(ty) <= (size_t)smem_max) return ty;
  return 0;
}

// One backward step (index n = 0, 1, ... in backward order).  fused (masked
// form): the kernel forms lambda^n from the previous step's accumulators
// over u_prev, and the accumulators rotate over three buffers (read n % 3,
// accumulate into (n + 1) % 3, zero (n + 2) % 3); otherwise lambda^n comes
// from lam, two buffers alternate, and the slope transpose writes
// lambda^{n+1} into lam_out.
template <typename T>
fk_status adj_step(fk_plan* p, int n, const void* u_in, const void* u_prev, bool fused,
                   const void* lam, void* lam_out, double* dth, int ty, cudaStream_t s) {
  AdjArgs<T> g;
  memset(&g, 0, sizeof(g));
  if (sizeof(T) == 4)
    fk_fill_step2d_f32(p, n, (Step2D<float>*)&g.s);
  else
    fk_fill_step2d_f64(p, n, (Step2D<double>*)&g.s);
  // the adjoint kernels stage the direct kernel's column-major layout,
  // whatever step kernel the forward march uses
  g.s.mode = 0;
  g.s.win = 0;
  g.s.hx = p->halo[0];
  g.s.hy = p->halo[1];
  g.s.lx = g.s.tx + 2 * g.s.hx + 2;
  g.s.ty = ty;
  g.s.ly = ty + 2 * g.s.hy + 2;
  g.s.lyr = g.s.ly | 1;
  g.s.u_in = (const T*)u_in;
  const int64_t J3 = 3 * p->J;
  T* mu_next = nullptr;
  if (fused) {
    g.lam = nullptr;
    g.mu = (T*)p->adj_mu + ((n + 1) % 3) * J3;
    g.mu_prev = (const T*)p->adj_mu + (n % 3) * J3;
    g.mu_clear = (T*)p->adj_mu + ((n + 2) % 3) * J3;
    g.u_prev = (const T*)u_prev;
  } else {
    // two mu buffers of 3 J values: step n accumulates into buffer n % 2
    // while its slope transpose clears the other one for step n + 1
    g.lam = (const T*)lam;
    g.mu = (T*)p->adj_mu + (n & 1) * J3;
    mu_next = (T*)p->adj_mu + ((n + 1) & 1) * J3;
  }
  g.dth = dth;
  const double tn = n * p->dt;
  if (p->coeffs.family == FK_CELLULAR_FLOW) {
    const double eps = p->coeffs.p[1], om = p->coeffs.p[2], D = p->coeffs.p[3];
    g.st = (T)sin(om * tn);
    g.sw = (T)(eps * tn * cos(om * tn));
    g.cn = (T)(D > 0.0 ? 1.0 / (2.0 * D) : 0.0);  // sigma = sqrt(2D): dsigma/dD / sigma
  } else {
    g.cbx = (T)(p->dt / p->h[0]);
    g.cby = (T)(p->dt / p->h[1]);
    g.cn = (T)(p->coeffs.p[3] > 0.0 ? 1.0 / p->coeffs.p[3] : 0.0);  // sigma = s
  }
  cudaError_t e;
  // fk_adjoint_kernel_times: an event pair around the backward-step kernel
  cudaEvent_t* ev = nullptr;
  if (p->adj_rec && p->adj_ev_used + 2 <= p->adj_ev_cap) {
    ev = p->adj_ev + p->adj_ev_used;
    p->adj_ev_used += 2;
    if (cudaEventRecord(ev[0], s) != cudaSuccess) return FK_ERR_CUDA;
  }
  if constexpr (sizeof(T) == 4) {
    if (adj_use_masked(p)) {
      // the masked window's layout: halo, row-major records, cell offsets
      g.s.mode = 2;
      g.s.win = p->mwin;
      g.s.hx = p->mhalo[0];
      g.s.hy = p->mhalo[1];
      g.s.lx = g.s.tx + 2 * g.s.hx + 2;
      g.s.ty = p->adj_ty;
      g.s.ly = g.s.ty + 2 * g.s.hy + 2;
      g.s.lyr = g.s.lx | 1;
      for (int q = 0; q < p->q; ++q) {
        g.s.wm[q] = p->mwm[q];
        g.s.wmf[q] = (T)p->mwm[q];
      }
      AdjArgs<float>& gf = (AdjArgs<float>&)g;
      gf.tab = (const float4*)p->adj_tab;
      for (int m = 0; m < 2; ++m) {
        for (int b = 0; b < FK_MAXQ_2D; ++b) gf.brk[m][b] = p->adj_break[m][b];
        gf.last[m] = p->adj_last[m];
      }
      e = launch_adj_masked(gf, p->q, s);
    } else {
      e = launch_adj<T>(g, p->q, s);
    }
  } else {
    e = launch_adj<T>(g, p->q, s);
  }
  if (e != cudaSuccess) return FK_ERR_CUDA;
  if (ev && cudaEventRecord(ev[1], s) != cudaSuccess) return FK_ERR_CUDA;
  if (fused) return FK_OK;
  const dim3 b(32, 8), gr((p->grid.n[0] + 31) / 32, (p->grid.n[1] + 7) / 8);
  k_adj_slopes_t<T><<<gr, b, 0, s>>>((const T*)u_in, (const T*)g.mu, (T*)lam_out, mu_next,
                                     p->grid.n[0], p->grid.n[1]);
  e = cudaGetLastError();
  return e == cudaSuccess ? FK_OK : FK_ERR_CUDA;
}

}  // namespace

extern "C" fk_status fk_adjoint(fk_plan* p, const void* u_terminal, const double* cotangent_u0,
                                double* dtheta, void* du_terminal, int K, cudaStream_t s) {
  FkRange range("fk_adjoint");
  if (!p || !cotangent_u0 || K < 1) return FK_ERR_INVALID_ARG;
  if (p->grid.dim != 2 || p->path != FK_PATH_MATRIX_FREE) return FK_ERR_UNSUPPORTED;
  // the parameter derivatives are those of the cellular flow or the constant
  // drift, on a uniform mesh of a box whose faces all absorb
  if (p->periodic_x || p->nu || p->coeffs.family == FK_PAPER_CELLULAR) return FK_ERR_UNSUPPORTED;
  const int N = p->n_steps;
  if (K > N) K = N;
  const int M = (N + K - 1) / K;  // checkpoints at n = 0, K, ..., and N
  const int64_t fb = p->J * p->elem;
  // tile height of the scatter kernel: the forward tile if its staging plus
  // the accumulators fit, else shorter
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  int ty = p->tile[1];
  while (ty > 8) {
    const int ly = ty + 2 * p->halo[1] + 2;
    if (adj_smem(32 + 2 * p->halo[0] + 2, ly, ly | 1, p->elem) + kAdjStatic <= (size_t)smem_max)
      break;
    ty -= 8;
  }
  {
    const int ly = ty + 2 * p->halo[1] + 2;
    if (adj_smem(32 + 2 * p->halo[0] + 2, ly, ly | 1, p->elem) + kAdjStatic > (size_t)smem_max)
      return FK_ERR_UNSUPPORTED;
  }
  p->adj_ty = adj_use_masked(p) ? adj_masked_ty(p, smem_max) : 0;
  if (adj_use_masked(p) && p->adj_ty == 0) return FK_ERR_UNSUPPORTED;
  p->adj_kernel = adj_use_masked(p) ? 2 : 1;
  if (adj_use_masked(p) && !p->adj_tab) {
    std::vector<float> tab;
    if (!adj_tables(p, tab)) return FK_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FK_ERR_CUDA;
    fk_status st = fk_dev_alloc(p, &p->adj_tab, tab.size() * sizeof(float));
    if (st != FK_OK) return st;
    if (cudaMemcpy(p->adj_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return FK_ERR_CUDA;
  }
  // the masked form forms lambda inside its kernel (three accumulator buffers)
  const bool fused = p->adj_kernel == 2 && p->adj_ty <= kAdjLamRows;
  // workspace: checkpoints (M+1), two segments (2K), lambda x2, mu (3 x 3 fields), dtheta
  const int64_t need = (int64_t)(M + 1 + 2 * K + 2 + 9) * fb + 64;
  if (p->adj_bytes < need) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return FK_ERR_CUDA;
    fk_dev_free(p->adj_ws);
    p->adj_ws = nullptr;
    p->adj_bytes = 0;
    fk_status st = fk_dev_alloc(p, &p->adj_ws, (size_t)need);
    if (st != FK_OK) return st;
    p->adj_bytes = need;
  }
  char* base = (char*)p->adj_ws;
  auto ckpt = [&](int m) { return (void*)(base + (int64_t)m * fb); };
  char* seg = base + (int64_t)(M + 1) * fb;  // segment buffers 0 and 1, K fields each
  char* rest = seg + (int64_t)(2 * K) * fb;
  void* lam[2] = {rest, rest + fb};
  p->adj_mu = rest + 2 * fb;
  double* dth = dtheta ? dtheta : (double*)(rest + (int64_t)11 * fb);
  auto slot = [&](int n) { return n == N ? M : n / K; };  // n == N or n % K == 0

  // forward pass with checkpoints
  {
    FkRange fwd_range("fk_adjoint forward pass");
    cudaError_t e;
    if (u_terminal)
      e = fk_launch_copy(ckpt(M), u_terminal, fb, s);
    else
      e = fk_launch_fill_chi(ckpt(M), 2, p->grid.n[0], p->grid.n[1], p->elem, s);
    if (e != cudaSuccess) return FK_ERR_CUDA;
    const void* src = ckpt(M);
    for (int n = N - 1; n >= 1; --n) {  // u^0 itself is not needed
      void* dst = (n % K == 0) ? ckpt(slot(n)) : lam[n & 1];
      fk_status st = fk_enqueue_step(p, n, src, dst, nullptr, s);
      if (st != FK_OK) return st;
      src = dst;
    }
  }
  if (cudaMemsetAsync(p->adj_mu, 0, (size_t)9 * fb, s) != cudaSuccess ||
      cudaMemsetAsync(dth, 0, 4 * sizeof(double), s) != cudaSuccess)
    return FK_ERR_CUDA;
  // lambda^0 = g (fused: as the u part of the accumulators step 0 reads, its
  // slope parts zero)
  int cur = 0;
  {
    const int blocks = (int)((p->J + 255) / 256 < 152 * 16 ? (p->J + 255) / 256 : 152 * 16);
    void* dst0 = fused ? p->adj_mu : lam[cur];
    if (p->prec == FK_FP32)
      k_cast_in<float><<<blocks, 256, 0, s>>>(cotangent_u0, (float*)dst0, p->J);
    else
      k_cast_in<double><<<blocks, 256, 0, s>>>(cotangent_u0, (double*)dst0, p->J);
    if (cudaGetLastError() != cudaSuccess) return FK_ERR_CUDA;
  }
  // events for the backward-step kernels (fk_adjoint_kernel_times)
  p->adj_ev_used = 0;
  if (p->adj_rec && p->adj_ev_cap < 2 * N) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return FK_ERR_CUDA;
    cudaEvent_t* grown = (cudaEvent_t*)realloc(p->adj_ev, sizeof(cudaEvent_t) * 2 * N);
    if (!grown) return FK_ERR_OOM;
    p->adj_ev = grown;
    while (p->adj_ev_cap < 2 * N) {
      if (cudaEventCreate(&p->adj_ev[p->adj_ev_cap]) != cudaSuccess) return FK_ERR_CUDA;
      ++p->adj_ev_cap;
    }
  }
  // The recompute of a segment depends only on its checkpoint, so it runs
  // on the plan's second stream, one segment ahead of the backward steps
  // on s, into the other of two segment buffers: the forward steps and the
  // backward kernels, which are bound by different units, share the SMs.
  // Events order it: segment m + 1 is recomputed after the forward pass and
  // after segment m - 1's backward steps have read that buffer; segment m's
  // backward steps start after its recompute.  (Without the stream or the
  // events, everything runs on s, one segment after the other.)
  if (!p->adj_s2 && cudaStreamCreateWithFlags(&p->adj_s2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    p->adj_s2 = nullptr;
  }
  while (p->adj_s2 && p->adj_sev_n < 5) {
    if (cudaEventCreateWithFlags(&p->adj_sev[p->adj_sev_n], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    ++p->adj_sev_n;
  }
  const bool two = p->adj_s2 && p->adj_sev_n == 5;
  cudaStream_t rs = two ? p->adj_s2 : s;  // the recompute's stream
  cudaEvent_t* ev_rec = p->adj_sev + 1;     // per buffer: recomputed
  cudaEvent_t* ev_bwd = p->adj_sev + 3;     // per buffer: backward steps done
  if (two && (cudaEventRecord(p->adj_sev[0], s) != cudaSuccess ||
              cudaStreamWaitEvent(rs, p->adj_sev[0], 0) != cudaSuccess))
    return FK_ERR_CUDA;
  auto segbuf = [&](int m) { return seg + (int64_t)(m & 1) * K * fb; };
  // recompute u^{top-1} .. u^{lo+1} of segment m into its buffer
  auto recompute = [&](int m) -> fk_status {
    const int lo = m * K, top = (m + 1) * K < N ? (m + 1) * K : N;
    if (two && m >= 2 && cudaStreamWaitEvent(rs, ev_bwd[m & 1], 0) != cudaSuccess)
      return FK_ERR_CUDA;
    const void* src = ckpt(slot(top));
    for (int n = top - 1; n >= lo + 1; --n) {
      void* dst = segbuf(m) + (int64_t)(n - lo - 1) * fb;
      fk_status st = fk_enqueue_step(p, n, src, dst, nullptr, rs);
      if (st != FK_OK) return st;
      src = dst;
    }
    if (two && cudaEventRecord(ev_rec[m & 1], rs) != cudaSuccess) return FK_ERR_CUDA;
    return FK_OK;
  };
  // backward over segments [mK, top)
  fk_status rst = recompute(0);
  if (rst != FK_OK) return rst;
  const void* u_prev = nullptr;  // the previous backward step's u_in
  for (int m = 0; m < M; ++m) {
    FkRange seg_range("fk_adjoint segment");
    const int lo = m * K, top = (m + 1) * K < N ? (m + 1) * K : N;
    if (two && m + 1 < M) {
      rst = recompute(m + 1);
      if (rst != FK_OK) return rst;
    }
    if (two && cudaStreamWaitEvent(s, ev_rec[m & 1], 0) != cudaSuccess) return FK_ERR_CUDA;
    for (int n = lo; n < top; ++n) {
      const void* u_in = (n + 1 == top) ? ckpt(slot(top))
                                        : (const void*)(segbuf(m) + (int64_t)(n - lo) * fb);
      const void* up = u_prev ? u_prev : u_in;  // (step 0: the slope parts are 0)
      fk_status st =
          p->prec == FK_FP32
              ? adj_step<float>(p, n, u_in, up, fused, lam[cur], lam[cur ^ 1], dth, ty, s)
              : adj_step<double>(p, n, u_in, up, fused, lam[cur], lam[cur ^ 1], dth, ty, s);
      if (st != FK_OK) return st;
      cur ^= 1;
      u_prev = u_in;
    }
    if (two && cudaEventRecord(ev_bwd[m & 1], s) != cudaSuccess) return FK_ERR_CUDA;
    if (!two && m + 1 < M) {
      rst = recompute(m + 1);
      if (rst != FK_OK) return rst;
    }
  }
  if (fused && du_terminal) {
    // lambda^N: the slope transpose of the last step's accumulators
    const dim3 b(32, 8), gr((p->grid.n[0] + 31) / 32, (p->grid.n[1] + 7) / 8);
    const int64_t J3 = 3 * p->J;
    k_adj_slopes_t<float><<<gr, b, 0, s>>>((const float*)u_prev,
                                           (const float*)p->adj_mu + (N % 3) * J3,
                                           (float*)lam[cur],
                                           (float*)p->adj_mu + ((N + 1) % 3) * J3,
                                           p->grid.n[0], p->grid.n[1]);
    if (cudaGetLastError() != cudaSuccess) return FK_ERR_CUDA;
  }
  if (du_terminal && fk_launch_copy(du_terminal, lam[cur], fb, s) != cudaSuccess) return FK_ERR_CUDA;
  return FK_OK;
}

extern "C" fk_status fk_adjoint_kernel_times(fk_plan* p, int record, double* kernel_ms,
                                             int* launches) {
  if (!p || (record != 0 && record != 1)) return FK_ERR_INVALID_ARG;
  if (kernel_ms) *kernel_ms = 0.0;
  if (launches) *launches = 0;
  double total = 0.0;
  const int pairs = p->adj_ev_used / 2;
  for (int i = 0; i < pairs; ++i) {
    float ms = 0.f;
    if (cudaEventSynchronize(p->adj_ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, p->adj_ev[2 * i], p->adj_ev[2 * i + 1]) != cudaSuccess)
      return FK_ERR_CUDA;
    total += ms;
  }
  if (kernel_ms) *kernel_ms = total;
  if (launches) *launches = pairs;
  p->adj_rec = record;
  return FK_OK;
}
