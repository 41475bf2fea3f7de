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
//    the slope of node 1 and node n-1 that of node n-2), and the held value
//    into u^n at every node of an absorbing face (Eq. (e3): 1, or the face's
//    exit value in the runaway model);
//  * k_step3d forms each updated node's 1D weights in registers and sums
//    the records of its window, read through L1/L2 (a warp's 32
//    consecutive x-nodes read overlapping, contiguous windows); with
//    per-node coefficients, only the planes, rows and cells its own points
//    reach, often far fewer than the W^3 the widest node needs.
// The runaway model's per-node drift and sigma (Eq. (ex32d): erf, four
// exponentials, square roots) go into a table of six values per node that
// k_step3d reads: k_coef3d fills it once per plan for the static model, and
// for the quench variant, whose constants depend on t_n, the record launch
// fills it before each step (k_rec_coef3d).
// Positions are taken relative to the node in cells: point p of axis m is
// at i_m + rel_p with rel_p = b_m dt / h_m + sigma_m sqrt(2 dt) a_p / h_m.
//
// The runaway-electron model of Sec. 4.3 (FK_RUNAWAY_3D, x = (p, xi, r))
// takes its drift and diagonal sigma per node (Eq. (ex32d)) and its own face
// rules: an exit through p = p_max takes 1, through p = p_min or the wall
// r = r_hi 0, and a point beyond a face of xi or r = r_lo is mirrored back
// into the box (those faces' nodes are updated like interior ones).  The
// mirror keeps the sum separable (it acts on one coordinate), and the two
// kinds of exit split each axis's dropped weight into E1_m and E0_m: a
// point takes 1 when any coordinate leaves through a value-1 face, so
//   u^n = sum_inside + 1 - prod_m (1 - E1_m).
//
// The kernels and their launchers are templates on the precision; the
// translation units fk_march3d_f32.cu and fk_march3d_f64.cu instantiate one
// precision each, so that the parallel build compiles them side by side.
#pragma once

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

// The value a node on an absorbing face holds (Eq. (e3)): 1 when one of
// its faces has exit value 1, else 0; -1 for a node the scheme updates.
template <typename T>
__device__ __forceinline__ T held_value(const Step3D<T>& a, int i, int j, int k) {
  const int at[3] = {i, j, k}, n3[3] = {a.nx, a.ny, a.nz};
  bool on = false, one = false;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
#pragma unroll
    for (int up = 0; up < 2; ++up) {
      const int rule = a.face[m][up];
      if (at[m] == (up ? n3[m] - 1 : 0) && rule != FK_FACE_REFLECT) {
        on = true;
        one = one || rule == FK_FACE_EXIT1;
      }
    }
  }
  return on ? (one ? T(1) : T(0)) : T(-1);
}

// The record and the held boundary value of node (i, j, k).
template <typename T>
__device__ __forceinline__ void rec3d_node(const Step3D<T>& a, int i, int j, int k) {
  const int64_t sy = a.nx, sz = (int64_t)a.nx * a.ny;
  const int64_t node = (int64_t)k * sz + (int64_t)j * sy + i;
  const T* u = a.u_in;
  // slope of Eq. (e300) along axis m at index idx (n nodes, stride st):
  // scaled by the cell on a uniform mesh, a raw derivative from the
  // divided differences over the actual spacings on a non-uniform one
  auto slope = [&](int m, int idx, int n, int64_t st) {
    const int c = idx < 1 ? 1 : (idx > n - 2 ? n - 2 : idx);
    const T* b = u + node + (int64_t)(c - idx) * st;
    const T um = b[-st], u0 = b[0], up = b[st];
    if (a.nu) {
      const T* x = a.xc[m];
      return pchip_fast((u0 - um) / (x[c] - x[c - 1]), (up - u0) / (x[c + 1] - x[c]));
    }
    return pchip_fast(u0 - um, up - u0);
  };
  V4<T> r;
  r.x = u[node];
  r.y = slope(0, i, a.nx, 1);
  r.z = slope(1, j, a.ny, sy);
  r.w = slope(2, k, a.nz, sz);
  a.rec[node] = r;
  const T held = held_value(a, i, j, k);
  if (held >= T(0)) {
    a.u_out[node] = held;
    if (a.snap) a.snap[node] = held;
  }
}

// Records and boundary values of one field.
template <typename T>
__global__ void __launch_bounds__(kRecThreads) k_rec3d(const Step3D<T> a) {
  const int i = blockIdx.x * kRecThreads + threadIdx.x;
  if (i >= a.nx) return;
  rec3d_node(a, i, (int)blockIdx.y, (int)blockIdx.z);
}

// Terminal indicator: 1 on the faces whose exit value is 1, 0 elsewhere.
template <typename T>
__global__ void __launch_bounds__(kRecThreads) k_chi3d(const Step3D<T> a, T* u) {
  const int i = blockIdx.x * kRecThreads + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= a.nx) return;
  const int at[3] = {i, j, k}, n3[3] = {a.nx, a.ny, a.nz};
  bool one = false;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    one = one || (at[m] == 0 && a.face[m][0] == FK_FACE_EXIT1) ||
          (at[m] == n3[m] - 1 && a.face[m][1] == FK_FACE_EXIT1);
  }
  u[((int64_t)k * a.ny + j) * a.nx + i] = one ? T(1) : T(0);
}

// The 1D weights of one axis over its window [org, org + W): node i of n,
// points at i + sh + gs a_q.  Returns the weight of the points that exit
// with value 1 (E1) and with value 0 (E0, the runaway faces only); with RE
// a point beyond a reflecting face is mirrored into the box first.  Sets
// bad when an inside point's cell falls outside the window (the plan's W
// rules this out; the check keeps every read in bounds regardless).  The
// slots that can carry weight are [tlo, thi] (empty, tlo > thi, when every
// point exits): W covers the widest spread on the mesh, and a node whose
// points spread less needs fewer of the window's records.
template <typename T, int W, bool RE>
__device__ __forceinline__ void axis_weights(const Step3D<T>& a, int m, int i, int n, T sh, T gs,
                                             T (&V)[W], T (&D)[W], T& E1, T& E0, int& org,
                                             int& tlo, int& thi, unsigned& bad) {
  tlo = W;
  thi = -1;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    V[t] = T(0);
    D[t] = T(0);
  }
  E1 = T(0);
  E0 = T(0);
  const T lo = T(-i), hi = T(n - 1 - i);  // the box, relative to the node
  // the abscissae ascend and gs >= 0: point 0 is the leftmost
  int o = i + (int)floor_t(sh + gs * a.ga[0]);
  o = o < 0 ? 0 : o;
  o = o > n - W ? n - W : o;
  org = o;
  int rlo = FK_FACE_EXIT1, rhi = FK_FACE_EXIT1;
  if constexpr (RE) {
    rlo = a.face[m][0];
    rhi = a.face[m][1];
  }
#pragma unroll
  for (int q = 0; q < FK_MAXQ_2D; ++q) {
    if (q < a.q) {
      T rel = sh + gs * a.ga[q];
      const T wq = a.gw[q];
      if constexpr (RE) {
        // mirror image in a reflecting face
        if (rel < lo && rlo == FK_FACE_REFLECT) rel = T(2) * lo - rel;
        if (rel > hi && rhi == FK_FACE_REFLECT) rel = T(2) * hi - rel;
      }
      const bool below = rel < lo, above = rel > hi;
      const bool in = !(below || above);
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
      const int rule = below ? rlo : rhi;
      E1 += (!in && rule == FK_FACE_EXIT1) ? wq : T(0);
      if constexpr (RE) E0 += (!in && rule == FK_FACE_EXIT0) ? wq : T(0);
      const T wi = (in && ok) ? wq : T(0);
      if (in && ok) {
        tlo = off < tlo ? off : tlo;
        thi = off + 1 > thi ? off + 1 : thi;
      }
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
}

// The same 1D weights on a non-uniform axis (node coordinates x[0..n-1]):
// points at x_i + sh + gs a_q in physical lengths (sh = b dt, gs = sigma
// sqrt(2 dt)), each located by walking from the node's cell (the last node
// at or left of the point, clamped to a cell, as the oracle's bisection
// finds it), the cell's own width scaling the slope basis (the records hold
// raw derivatives).  The window starts at the lowest cell an inside point
// reaches (mirrored points included), clamped to [0, n - W].
template <typename T, int W, bool RE>
__device__ __forceinline__ void axis_weights_nu(const Step3D<T>& a, int m, int i, int n, T sh,
                                                T gs, T (&V)[W], T (&D)[W], T& E1, T& E0,
                                                int& org, int& tlo, int& thi, unsigned& bad) {
  const T* __restrict__ x = a.xc[m];
#pragma unroll
  for (int t = 0; t < W; ++t) {
    V[t] = T(0);
    D[t] = T(0);
  }
  E1 = T(0);
  E0 = T(0);
  tlo = W;
  thi = -1;
  const T lo = x[0], hi = x[n - 1], xi = x[i];
  int rlo = FK_FACE_EXIT1, rhi = FK_FACE_EXIT1;
  if constexpr (RE) {
    rlo = a.face[m][0];
    rhi = a.face[m][1];
  }
  T z[FK_MAXQ_2D];
  int cq[FK_MAXQ_2D];
  int cmin = n;
#pragma unroll
  for (int q = 0; q < FK_MAXQ_2D; ++q) {
    if (q < a.q) {
      T v = xi + sh + gs * a.ga[q];
      if constexpr (RE) {
        if (v < lo && rlo == FK_FACE_REFLECT) v = T(2) * lo - v;
        if (v > hi && rhi == FK_FACE_REFLECT) v = T(2) * hi - v;
      }
      int c = i < n - 2 ? i : n - 2;
      while (c > 0 && x[c] > v) --c;
      while (c < n - 2 && x[c + 1] <= v) ++c;
      z[q] = v;
      cq[q] = c;
      if (!(v < lo || v > hi)) cmin = c < cmin ? c : cmin;
    }
  }
  int o = cmin > n - W ? n - W : cmin;
  o = o < 0 ? 0 : o;
  org = o;
#pragma unroll
  for (int q = 0; q < FK_MAXQ_2D; ++q) {
    if (q < a.q) {
      const T v = z[q];
      const T wq = a.gw[q];
      const bool below = v < lo, above = v > hi;
      const bool in = !(below || above);
      const int c = cq[q];
      const T h = x[c + 1] - x[c];
      const T s = (v - x[c]) / h;
      const int off = c - o;
      const bool ok = off >= 0 && off <= W - 2;
      if (in && !ok) bad = 1u;
      const int rule = below ? rlo : rhi;
      E1 += (!in && rule == FK_FACE_EXIT1) ? wq : T(0);
      if constexpr (RE) E0 += (!in && rule == FK_FACE_EXIT0) ? wq : T(0);
      const T wi = (in && ok) ? wq : T(0);
      if (in && ok) {
        tlo = off < tlo ? off : tlo;
        thi = off + 1 > thi ? off + 1 : thi;
      }
      const T s2 = s * s, r1 = T(1) - s;
      const T h00 = (T(1) + T(2) * s) * r1 * r1, h01 = s2 * (T(3) - T(2) * s);
      const T h10 = h * (s * r1 * r1), h11 = -h * (s2 * r1);
#pragma unroll
      for (int t = 0; t < W; ++t) {
        V[t] += (t == off) ? wi * h00 : ((t == off + 1) ? wi * h01 : T(0));
        D[t] += (t == off) ? wi * h10 : ((t == off + 1) ? wi * h11 : T(0));
      }
    }
  }
}

// Entry t of a register array indexed by a runtime value (a select per
// entry keeps the array in registers).
template <int W, typename T>
__device__ __forceinline__ T pick(const T (&v)[W], int t) {
  T r = v[0];
#pragma unroll
  for (int e = 1; e < W; ++e) r = (e == t) ? v[e] : r;
  return r;
}

template <typename T>
__device__ __forceinline__ T erf_t(T x);
template <>
__device__ __forceinline__ float erf_t<float>(float x) { return erff(x); }
template <>
__device__ __forceinline__ double erf_t<double>(double x) { return erf(x); }

// Drift and diagonal sigma of the runaway-electron model at node (i, j, k)
// (Eq. (ex32d) of Sec. 4.3), returned as the point shift sh = b dt / h and
// scale gs = sigma sqrt(2 dt) / h per axis, in cells (NU: physical lengths
// b dt and sigma sqrt(2 dt), at the plan's FP64 node coordinates).  Collision functions
// C_A = nu v_T^2 psi(y)/y, C_B = (nu v_T^2 / 2y)[Z + phi(y) - psi(y) +
// y^2 delta^4 / 2], C_F = 2 nu v_T psi(y) with phi = erf, psi(y) =
// (phi - y phi') / (2 y^2), y = p / gamma, gamma = sqrt(1 + (delta p)^2);
// the p drift carries (1/p^2) d/dp (p^2 C_A) by the chain rule (dy/dp =
// 1/gamma^3, psi' = phi' - 2 psi / y).  The node coordinates are formed in
// FP64 without contraction, and the step V(r) = V_0 1{r > r_D} is decided
// there; the rest runs in T.
template <typename T, bool NU>
__device__ __forceinline__ void runaway_coef(const Step3D<T>& a, int i, int j, int k, T (&sh)[3],
                                             T (&gs)[3]) {
  double xp, xx, xr;
  if constexpr (NU) {  // the FP64 node coordinates of the plan
    xp = a.xd[0][i];
    xx = a.xd[1][j];
    xr = a.xd[2][k];
  } else {
    xp = __dadd_rn(a.lo[0], __dmul_rn((double)i, a.h[0]));
    xx = __dadd_rn(a.lo[1], __dmul_rn((double)j, a.h[1]));
    xr = __dadd_rn(a.lo[2], __dmul_rn((double)k, a.h[2]));
  }
  const bool beyond = xr > a.rp[6];
  const T mom = (T)xp, xi = (T)xx, r = (T)xr;
  const T E = (T)a.rp[0], tau = (T)a.rp[1], Z = (T)a.rp[2], delta = (T)a.rp[3];
  const T nu = (T)a.rp[4], vT = (T)a.rp[5], rD = (T)a.rp[6], Wr = (T)a.rp[7];
  const T Dp = (T)a.rp[8], V0 = (T)a.rp[9], D0 = (T)a.rp[10];
  const T dm = delta * mom;
  const T gam = sqrt(T(1) + dm * dm);
  const T y = mom / gam;
  const T phi = erf_t(y);
  const T dphi = T(1.1283791670955126) * exp(-y * y);  // 2 / sqrt(pi) exp(-y^2)
  const T psi = (phi - y * dphi) / (T(2) * y * y);
  const T dpsi = dphi - T(2) * psi / y;
  const T nv2 = nu * vT * vT;
  const T CA = nv2 * psi / y;
  const T d2 = delta * delta;
  const T CB = T(0.5) * nv2 / y * (Z + phi - psi + T(0.5) * y * y * (d2 * d2));
  const T CF = T(2) * nu * vT * psi;
  const T dy = T(1) / (gam * gam * gam);
  const T df = T(2) * mom * psi / y + mom * mom * (dpsi / y - psi / (y * y)) * dy;
  const T om = T(1) - xi * xi;
  const T b0 = E * xi - gam * mom / tau * om - CF + nv2 * df / (mom * mom);
  const T b1 = E * om / mom - xi * om / (tau * gam) - T(2) * xi * CB / (mom * mom);
  // 1 + tanh z = 2 / (1 + e^{-2z}) and 1 - tanh z = 2 / (1 + e^{2z}): no
  // cancellation where tanh is near -1 (in FP32, 1 + tanhf(-10) is 0, which
  // would drop a radial diffusion that FP64 keeps)
  const T z = (r - rD) / Wr;
  const T onep = T(2) / (T(1) + exp(T(-2) * z)), onem = T(2) / (T(1) + exp(T(2) * z));
  const T q = mom / Dp;
  const T ep = exp(-q * q);
  const T Dr = T(0.5) * D0 * onep * ep;
  const T b2 = (beyond ? V0 : T(0)) + T(0.5) * D0 * onep * onem / Wr * ep;
  const T s0 = sqrt(T(2) * CA);
  const T s1 = sqrt(T(2) * CB) * sqrt(om > T(0) ? om : T(0)) / mom;
  const T s2 = sqrt(T(2) * Dr);
  const T b[3] = {b0, b1, b2}, sg[3] = {s0, s1, s2};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    if constexpr (NU) {  // physical lengths
      sh[m] = b[m] * a.dt;
      gs[m] = sg[m] * a.sq2dt;
    } else {
      sh[m] = b[m] * a.dt / (T)a.h[m];
      gs[m] = sg[m] * a.sq2dt / (T)a.h[m];
    }
  }
}

// Resident CTAs per SM that k_step3d's register budget is set for.  FP32,
// measured on a GB300 against the unbounded budget (132 registers at W = 8):
// 4 for the wide uniform windows (the 97 x 65 x 41 runaway march 209 ->
// 177 ms, the 129^3 constant drift 263 -> 223 ms), 5 for W <= 6 and
// non-uniform axes (quench 332 -> 318 ms, the 97 x 65 x 128 non-uniform
// runaway march 738 -> 664 ms), a few spilled bytes at most.  FP64 keeps
// the compiler's budget.
template <typename T, int W, bool NU>
constexpr int step3d_min_blocks() {
  return sizeof(T) == 8 ? 1 : (NU || W <= 6) ? 5 : 4;
}

template <typename T, int W, bool RE, bool NU>
__global__ void __launch_bounds__(kRecThreads, (step3d_min_blocks<T, W, NU>()))
    k_step3d(const Step3D<T> a) {
  const int i = a.first[0] + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = a.first[1] + blockIdx.y, k = a.first[2] + blockIdx.z;
  if (i >= a.first[0] + a.count[0]) return;
  const int64_t sy = a.nx, sz = (int64_t)a.nx * a.ny;
  const int64_t node = (int64_t)k * sz + (int64_t)j * sy + i;

  // shift and scale of the points per axis, in cells: plan constants for
  // the constant drift, per node for the runaway model
  T sh[3], gs[3];
  if constexpr (RE) {  // k_coef3d's table (once per plan, or this step's for the quench)
    const int64_t J = sz * a.nz;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      sh[m] = a.coef[m * J + node];
      gs[m] = a.coef[(3 + m) * J + node];
    }
  } else {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      sh[m] = a.cd[m];
      gs[m] = a.gs[m];
    }
  }

  // 1D weights per axis
  T Vx[W], Dx[W], Vy[W], Dy[W], Vz[W], Dz[W];
  T E1x, E0x, E1y, E0y, E1z, E0z;
  int ox, oy, oz, xlo, xhi, ylo, yhi, zlo, zhi;
  unsigned bad = 0;
  if constexpr (NU) {
    axis_weights_nu<T, W, RE>(a, 0, i, a.nx, sh[0], gs[0], Vx, Dx, E1x, E0x, ox, xlo, xhi, bad);
    axis_weights_nu<T, W, RE>(a, 1, j, a.ny, sh[1], gs[1], Vy, Dy, E1y, E0y, oy, ylo, yhi, bad);
    axis_weights_nu<T, W, RE>(a, 2, k, a.nz, sh[2], gs[2], Vz, Dz, E1z, E0z, oz, zlo, zhi, bad);
  } else {
    axis_weights<T, W, RE>(a, 0, i, a.nx, sh[0], gs[0], Vx, Dx, E1x, E0x, ox, xlo, xhi, bad);
    axis_weights<T, W, RE>(a, 1, j, a.ny, sh[1], gs[1], Vy, Dy, E1y, E0y, oy, ylo, yhi, bad);
    axis_weights<T, W, RE>(a, 2, k, a.nz, sh[2], gs[2], Vz, Dz, E1z, E0z, oz, zlo, zhi, bad);
  }

  const V4<T>* R = a.rec;
  const T uj = R[node].x;
  // one plane c of the window: its W x W records against the x and y
  // weights.  With per-node coefficients (RE) only the rows [ylo, yhi] and
  // cells [xlo, xhi] that can carry weight are read (the others would add
  // exact zeros); with constant coefficients every node reaches the whole
  // window, and the unconditional loops schedule better.
  auto plane_sum = [&](int c, T vz, T dz) {
    const V4<T>* plane = R + (int64_t)(oz + c) * sz + (int64_t)oy * sy + ox;
    T P = T(0), Pz = T(0);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      if ((RE || NU) && (b < ylo || b > yhi)) continue;
      const V4<T>* row = plane + (int64_t)b * sy;
      T s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
      for (int t = 0; t < W; ++t) {
        if (!(RE || NU) || (t >= xlo && t <= xhi)) {
          const V4<T> r = row[t];
          s1 += Vx[t] * (r.x - uj) + Dx[t] * r.y;
          s2 += Vx[t] * r.z;
          s3 += Vx[t] * r.w;
        }
      }
      P += Vy[b] * s1 + Dy[b] * s2;
      Pz += Vy[b] * s3;
    }
    return vz * P + dz * Pz;
  };
  T acc = T(0);
  if constexpr (RE || NU) {
    // planes in a loop over the reached ones (the runaway instantiations
    // would double the build time if unrolled as well)
#pragma unroll 1
    for (int c = zlo; c <= zhi; ++c) acc += plane_sum(c, pick<W>(Vz, c), pick<W>(Dz, c));
  } else {
#pragma unroll
    for (int c = 0; c < W; ++c) acc += plane_sum(c, Vz[c], Dz[c]);
  }
  // value-1 exit mass 1 - (1 - E1x)(1 - E1y)(1 - E1z), exactly 0 when no
  // point exits; the window part is u_j + sum w (Itilde - u_j) over the
  // inside points, whose weight is (1 - Ex)(1 - Ey)(1 - Ez)
  const T ex1 = E1x + (T(1) - E1x) * (E1y + (T(1) - E1y) * E1z);
  T un;
  if constexpr (RE) {
    const T Ex = E1x + E0x, Ey = E1y + E0y, Ez = E1z + E0z;
    const T exall = Ex + (T(1) - Ex) * (Ey + (T(1) - Ey) * Ez);
    un = uj + acc + (ex1 - uj * exall);
  } else {
    un = uj + acc + (T(1) - uj) * ex1;
  }
  a.u_out[node] = un;
  if (a.snap) a.snap[node] = un;
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// The runaway coefficients of every node k_step3d updates, once per plan
// (the static model's do not depend on t).
template <typename T, bool NU>
__global__ void __launch_bounds__(kRecThreads) k_coef3d(const Step3D<T> a, T* coef) {
  const int i = a.first[0] + blockIdx.x * blockDim.x + threadIdx.x;
  const int j = a.first[1] + blockIdx.y, k = a.first[2] + blockIdx.z;
  if (i >= a.first[0] + a.count[0]) return;
  const int64_t J = (int64_t)a.nx * a.ny * a.nz;
  const int64_t node = ((int64_t)k * a.ny + j) * a.nx + i;
  T sh[3], gs[3];
  runaway_coef<T, NU>(a, i, j, k, sh, gs);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    coef[m * J + node] = sh[m];
    coef[(3 + m) * J + node] = gs[m];
  }
}

// The quench variant's step prologue in one launch: the records (as
// k_rec3d) and, at the nodes the step updates, the coefficients of t_n (as
// k_coef3d); two launches before.
template <typename T, bool NU>
__global__ void __launch_bounds__(kRecThreads) k_rec_coef3d(const Step3D<T> a, T* coef) {
  const int i = blockIdx.x * kRecThreads + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  if (i >= a.nx) return;
  rec3d_node(a, i, j, k);
  if (i < a.first[0] || i >= a.first[0] + a.count[0] || j < a.first[1] ||
      j >= a.first[1] + a.count[1] || k < a.first[2] || k >= a.first[2] + a.count[2])
    return;
  const int64_t J = (int64_t)a.nx * a.ny * a.nz;
  const int64_t node = ((int64_t)k * a.ny + j) * a.nx + i;
  T sh[3], gs[3];
  runaway_coef<T, NU>(a, i, j, k, sh, gs);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    coef[m * J + node] = sh[m];
    coef[(3 + m) * J + node] = gs[m];
  }
}

template <typename T, int W>
cudaError_t launch_w(const Step3D<T>& a, cudaStream_t s) {
  const int in = a.count[0];
  const int bx = in <= 32 ? 32 : (in <= 64 ? 64 : kRecThreads);
  const dim3 grid((unsigned)((in + bx - 1) / bx), (unsigned)a.count[1], (unsigned)a.count[2]);
  const bool re = a.family == FK_RUNAWAY_3D;
  if (a.nu) {
    if (re)
      k_step3d<T, W, true, true><<<grid, bx, 0, s>>>(a);
    else
      k_step3d<T, W, false, true><<<grid, bx, 0, s>>>(a);
  } else if (re) {
    k_step3d<T, W, true, false><<<grid, bx, 0, s>>>(a);
  } else {
    k_step3d<T, W, false, false><<<grid, bx, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t fk_launch_step3d(const Step3D<T>& a, cudaStream_t s) {
  {
    const dim3 grid((unsigned)((a.nx + kRecThreads - 1) / kRecThreads), (unsigned)a.ny,
                    (unsigned)a.nz);
    if (a.family == FK_RUNAWAY_3D && a.coef_per_step) {
      T* coef = const_cast<T*>(a.coef);
      if (a.nu)
        k_rec_coef3d<T, true><<<grid, kRecThreads, 0, s>>>(a, coef);
      else
        k_rec_coef3d<T, false><<<grid, kRecThreads, 0, s>>>(a, coef);
    } else {
      k_rec3d<T><<<grid, kRecThreads, 0, s>>>(a);
    }
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

template <typename T>
cudaError_t fk_launch_coef3d(const Step3D<T>& a, T* coef, cudaStream_t s) {
  const dim3 grid((unsigned)((a.count[0] + kRecThreads - 1) / kRecThreads), (unsigned)a.count[1],
                  (unsigned)a.count[2]);
  if (a.nu)
    k_coef3d<T, true><<<grid, kRecThreads, 0, s>>>(a, coef);
  else
    k_coef3d<T, false><<<grid, kRecThreads, 0, s>>>(a, coef);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fk_launch_chi3d(const Step3D<T>& a, T* u, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nx + kRecThreads - 1) / kRecThreads), (unsigned)a.ny,
                  (unsigned)a.nz);
  k_chi3d<T><<<grid, kRecThreads, 0, s>>>(a, u);
  return cudaGetLastError();
}
