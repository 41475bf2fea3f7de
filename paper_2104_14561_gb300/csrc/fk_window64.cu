// Masked tensor-window step of Scheme 1 (Sec. 3.1.5) in FP64, for sm_103a.
//
// The factorisation of the FP32 kernel (fk_window.cuh): for node j the
// tensor Gauss-Hermite points of Eq. (e31) are X_p x Y_q (drift and sigma
// at the node), so with the zero-twist Hermite interpolant of Eq. (Lag11)
//
//   u^n_j = u_j + sum_{c,r} [(u_{c,r} - u_j) phi_c Phi_r + h u_x(c,r) psi_c Phi_r
//                            + h u_y(c,r) phi_c Psi_r]  +  (1 - u_j)(E_x + E_y - E_x E_y)
//
// over a W x W node window, with 1D weights from the points that stay in the
// box and the dropped (exiting) weight E per axis (Eq. (e24)).  The FP64
// pipe of this part is the limit, so the form is chosen to spend few FP64
// operations: W^2 cells x 4 plus 2Q 1D points x about 20, against Q^2
// points x (12 corner terms + the bicubic basis) in the direct kernel.
//
// Per CTA (32 x ty output nodes): u^{n+1} over the tile plus halo is staged
// with cp.async into the first half of each 16-byte record, the slopes of
// Eq. (e300) complete the records {u, h u_x} and {h u_y} in place, then one
// node per thread and pass.  The point weights use the plan's cell-offset
// pattern, compiled in (fk_mpat), and pick each point's cell pair with
// selects rather than FP64 multiplies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {

// Records of the staged tile (lx x ly nodes, row pitch lx): R[r][c] =
// {u_c, h u_x(c)} and Yh[r][c] = h u_y(c) for staged nodes 1..lx-2 x
// 1..ly-2 (u alone elsewhere, zero outside the mesh).  The end rule after
// Eq. (e300) gives node 0 the slope of node 1 and node n-1 that of node n-2:
// an end column takes its x-differences one column inwards, and the end rows
// copy the y-slopes of their neighbour row afterwards.
template <bool MF>
__device__ __forceinline__ void stage_rec64(const Step2D<double>& a, double2* R, double* Yh,
                                            int gi0, int gk0) {
  const int lx = a.lx, ly = a.ly;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const uint32_t sR = (uint32_t)__cvta_generic_to_shared(R);
    const double* base = field_in<MF>(a);
#pragma unroll 1
    for (int r = warp; r < ly; r += FK_THREADS / 32) {
      const int gk = gk0 + r;
      const bool rowin = (unsigned)gk < (unsigned)a.ny;
      const double* src = base + (int64_t)min(max(gk, 0), a.ny - 1) * a.nx;
      const uint32_t drow = sR + (uint32_t)(r * lx) * 16u;
      for (int c = lane; c < lx; c += 32) {
        const int g = gi0 + c;
        const bool in = rowin && (unsigned)g < (unsigned)a.nx;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(drow + 16u * c),
                     "l"(src + min(max(g, 0), a.nx - 1)), "r"(in ? 8 : 0));
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
  }
  // vertical sweeps: thread t owns column 1 + t % (lx-2) and a segment of
  // rows, carrying u of the rows above and below in registers.  Rewriting a
  // record keeps its u, so a neighbour reading that u meanwhile sees the same
  // value.
  {
    const int hc = lx - 2, hr = ly - 2;
    const int nseg = FK_THREADS / hc;
    const int seg = tid / hc, c = 1 + (tid - seg * hc);
    if (seg < nseg) {
      const int len = (hr + nseg - 1) / nseg;
      const int r0 = 1 + seg * len, r1 = min(r0 + len, hr + 1);
      const int gi = gi0 + c;
      const int ax = c + (gi == 0) - (gi == a.nx - 1);
      double up = r0 <= hr ? R[(r0 - 1) * lx + c].x : 0.0;
      double uc = r0 <= hr ? R[r0 * lx + c].x : 0.0;
      for (int r = r0; r < r1; ++r) {
        const double un = R[(r + 1) * lx + c].x;
        const double2* rx = R + r * lx + ax;
        const double X = pchip_scaled(rx[0].x - rx[-1].x, rx[1].x - rx[0].x);
        const double Y = pchip_scaled(uc - up, un - uc);
        R[r * lx + c] = make_double2(uc, X);
        Yh[r * lx + c] = Y;
        up = uc;
        uc = un;
      }
    }
    __syncthreads();
    const int rb = -gk0, rt = a.ny - 1 - gk0;
    const bool fb = rb >= 1 && rb <= hr - 1, ft = rt >= 2 && rt <= hr;
    if (fb || ft) {
      for (int e = tid; e < hc; e += FK_THREADS) {
        if (fb) Yh[rb * lx + 1 + e] = Yh[(rb + 1) * lx + 1 + e];
        if (ft) Yh[rt * lx + 1 + e] = Yh[(rt - 1) * lx + 1 + e];
      }
      __syncthreads();
    }
  }
}

__host__ __device__ constexpr int first_point64(int Q, int W, int K, int s) {
  for (int q = 0; q < Q; ++q)
    if (fk_mpat(Q, W, K, q) <= s && s <= fk_mpat(Q, W, K, q) + 2) return q;
  return Q;
}

template <bool FIRST>
__device__ __forceinline__ void put(double& slot, double v) {
  if constexpr (FIRST) slot = v;
  else slot += v;
}

// 1D weights of one axis from points q .. Q-1 of pattern K: PH[s] = phi_s,
// PS[s] = psi_s.  G[q] = g_q - m_q, w[q] the weights (shared memory), Z the
// drift after the window origin (point q sits at Z + G[q] + m_q); with EXIT
// a point outside [LO, HI] is dropped and its weight added to E.
template <int Q, int W, int K, bool EXIT, int q>
struct AxisWeights {
  __device__ __forceinline__ static void run(const double* G, const double* w, double Z,
                                             double LO, double HI, double (&PH)[W],
                                             double (&PS)[W], double& E) {
    if constexpr (q < Q) {
      constexpr int M = fk_mpat(Q, W, K, q);
      static_assert(M >= 0 && M + 2 < W, "pattern slot outside the window");
      const double tp = Z + G[q];
      double wq = w[q];
      if constexpr (EXIT) {
        const double sq = tp + (double)M;
        const bool out = sq < LO || sq > HI;
        E += out ? wq : 0.0;
        wq = out ? 0.0 : wq;
      }
      // (tp may round a hair outside [0, 2) at a cell face: the cubic is
      // continuous there, so the compare only has to pick one of the cells)
      const bool up = tp >= 1.0;
      const double t = up ? tp - 1.0 : tp;
      const double tt = t * t, om = t - 1.0;
      const double v1 = wq * (tt * fma(-2.0, t, 3.0));
      const double v0 = wq - v1;
      const double wto = (wq * t) * om;
      const double s0 = wto * om, s1 = wto * t;
      constexpr bool F0 = first_point64(Q, W, K, M) == q, F1 = first_point64(Q, W, K, M + 1) == q,
                     F2 = first_point64(Q, W, K, M + 2) == q;
      // the pair of cell nodes (M, M+1), or (M+1, M+2) one cell up
      put<F0>(PH[M], up ? 0.0 : v0);
      put<F1>(PH[M + 1], up ? v0 : v1);
      put<F2>(PH[M + 2], up ? v1 : 0.0);
      put<F0>(PS[M], up ? 0.0 : s0);
      put<F1>(PS[M + 1], up ? s0 : s1);
      put<F2>(PS[M + 2], up ? s1 : 0.0);
      AxisWeights<Q, W, K, EXIT, q + 1>::run(G, w, Z, LO, HI, PH, PS, E);
    }
  }
};

template <int Q, int W, int K>
__device__ __forceinline__ void weights64(int pat, bool exits, const double* GX, const double* GY,
                                          const double* w, double Zx, double Zy, double LOx,
                                          double HIx, double LOy, double HIy, double (&PX)[W],
                                          double (&SX)[W], double (&PY)[W], double (&SY)[W],
                                          double& Ex, double& Ey) {
  if constexpr (K < fk_npat(Q, W)) {
    if (pat == K) {
      if (exits) {
        AxisWeights<Q, W, K, true, 0>::run(GX, w, Zx, LOx, HIx, PX, SX, Ex);
        AxisWeights<Q, W, K, true, 0>::run(GY, w, Zy, LOy, HIy, PY, SY, Ey);
      } else {
        AxisWeights<Q, W, K, false, 0>::run(GX, w, Zx, LOx, HIx, PX, SX, Ex);
        AxisWeights<Q, W, K, false, 0>::run(GY, w, Zy, LOy, HIy, PY, SY, Ey);
      }
    } else {
      weights64<Q, W, K + 1>(pat, exits, GX, GY, w, Zx, Zy, LOx, HIx, LOy, HIy, PX, SX, PY, SY,
                             Ex, Ey);
    }
  }
}

// MF: several fields per launch (blockIdx.z), for Algorithm 1.
template <int Q, int W, bool MF>
__global__ void __launch_bounds__(FK_THREADS, 2) k_step2dm64(const Step2D<double> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx, ly = a.ly;
  double* GX = reinterpret_cast<double*>(smem);  // g_q - m_q per axis, w_q
  double* GY = GX + FK_MAXQ_2D;
  double* WQ = GY + FK_MAXQ_2D;
  double2* R = reinterpret_cast<double2*>(WQ + FK_MAXQ_2D);
  double* Yh = reinterpret_cast<double*>(R + ly * lx);
  const int tid = threadIdx.x;
  if (tid < Q) {
    GX[tid] = a.gmx[tid];
    GY[tid] = a.gmy[tid];
    WQ[tid] = a.w[tid];
  }
  const int i0 = 1 + blockIdx.x * 32, k0 = 1 + blockIdx.y * a.ty;
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;
  stage_rec64<MF>(a, R, Yh, gi0, gk0);

  const int lane = tid & 31, warp = tid >> 5;
  const int i = i0 + lane;
  if (i > a.nx - 2) return;
  const int li = i - gi0;
  const bool xsafe = i0 - a.hx >= 0 && i0 + 31 + a.hx <= a.nx - 1;
  double fcx = 1.0, fcy = 1.0;
  if (a.family == FK_CELLULAR_FLOW) {
    const double* ct = a.col_tab + 4 * (int64_t)i;
    fcx = a.A * ct[0] + a.e1 * ct[1];
    fcy = a.A * ct[2] + a.e2 * ct[3];
  }
  unsigned bad = 0;
#pragma unroll 1
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (k > a.ny - 2) break;
    const int lk = k - gk0;
    const double uj = R[lk * lx + li].x;
    double dx, dy;
    if (a.family == FK_CELLULAR_FLOW) {
      const double* rt = a.row_tab + 2 * (int64_t)k;
      dx = a.kx * rt[0] * fcx;
      dy = a.ky * rt[1] * fcy;
    } else {
      dx = a.cdx * fcx;
      dy = a.cdy * fcy;
    }
    // window origin: the cell of point 0 on each axis; positions after it
    // are Z + g_q with Z = D - F0
    const double fx0 = floor(dx + a.gx[0]), fy0 = floor(dy + a.gy[0]);
    int wx = li + (int)fx0, wy = lk + (int)fy0;
    if (wx < 1 || wx + W - 1 > lx - 2 || wy < 1 || wy + W - 1 > ly - 2) {
      bad = 1u;  // halo too small for this drift: flag, read an in-range window
      wx = 1;
      wy = 1;
    }
    const bool exits = !(xsafe && k - a.hy >= 0 && k + a.hy <= a.ny - 1);
    double PX[W], SX[W], PY[W], SY[W];
    double Ex = 0.0, Ey = 0.0;
    weights64<Q, W, 0>(a.mpat, exits, GX, GY, WQ, dx - fx0, dy - fy0, -(double)i - fx0,
                       (double)(a.nx - 1 - i) - fx0, -(double)k - fy0,
                       (double)(a.ny - 1 - k) - fy0, PX, SX, PY, SY, Ex, Ey);
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const double2* rr = R + (wy + r) * lx + wx;
      const double* yr = Yh + (wy + r) * lx + wx;
      double AE = 0.0, AX = 0.0, B = 0.0;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const double2 v = rr[c];
        AE = fma(PX[c], v.x - uj, AE);
        AX = fma(SX[c], v.y, AX);
        B = fma(PX[c], yr[c], B);
      }
      acc = fma(PY[r], AE + AX, fma(SY[r], B, acc));
    }
    const double ext = (1.0 - uj) * (Ex + Ey - Ex * Ey);
    const double un = uj + (acc + ext);
    const int64_t j = (int64_t)k * a.nx + i;
    field_out<MF>(a)[j] = un;
    if (a.snap) a.snap[j] = un;
    write_adjacent_boundary<MF>(a, i, k);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

template <int Q, int W>
cudaError_t launch_m64(const Step2D<double>& a, cudaStream_t s) {
  const size_t smem = fk_step2dm64_smem(a.ly, a.lx);
  const int nf = a.ncols > 1 ? a.ncols : 1;
  dim3 grid((a.nx - 2 + 31) / 32, (a.ny - 2 + a.ty - 1) / a.ty, nf);
  if (nf > 1)
    k_step2dm64<Q, W, true><<<grid, FK_THREADS, smem, s>>>(a);
  else
    k_step2dm64<Q, W, false><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int Q, int W>
cudaError_t attr_m64() {
  const int big = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_step2dm64<Q, W, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step2dm64<Q, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             big);
  return e;
}

template <int Q>
cudaError_t launch_q64(const Step2D<double>& a, cudaStream_t s) {
  switch (a.win) {
    case 3: return launch_m64<Q, 3>(a, s);
    case 4: return launch_m64<Q, 4>(a, s);
    case 5: return launch_m64<Q, 5>(a, s);
    case 6: return launch_m64<Q, 6>(a, s);
    case 7: return launch_m64<Q, 7>(a, s);
    case 8: return launch_m64<Q, 8>(a, s);
    case 9: return launch_m64<Q, 9>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int Q>
cudaError_t prepare_q64() {
  cudaError_t e = attr_m64<Q, 3>();
  if (e == cudaSuccess) e = attr_m64<Q, 4>();
  if (e == cudaSuccess) e = attr_m64<Q, 5>();
  if (e == cudaSuccess) e = attr_m64<Q, 6>();
  if (e == cudaSuccess) e = attr_m64<Q, 7>();
  if (e == cudaSuccess) e = attr_m64<Q, 8>();
  if (e == cudaSuccess) e = attr_m64<Q, 9>();
  return e;
}

}  // namespace

size_t fk_step2dm64_smem(int ly, int lx) {
  // point constants (3 x FK_MAXQ_2D doubles), then 16 + 8 bytes per staged node
  return (size_t)3 * FK_MAXQ_2D * 8 + (size_t)ly * lx * (16 + 8);
}

cudaError_t fk_launch_step2dm64(const Step2D<double>& a, int q, cudaStream_t s) {
  switch (q) {
    case 4: return launch_q64<4>(a, s);
    case 6: return launch_q64<6>(a, s);
    case 8: return launch_q64<8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fk_prepare_masked64(int q) {
  switch (q) {
    case 4: return prepare_q64<4>();
    case 6: return prepare_q64<6>();
    case 8: return prepare_q64<8>();
    default: return cudaSuccess;
  }
}
