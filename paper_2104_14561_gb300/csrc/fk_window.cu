// Masked tensor-window step of Scheme 1 (Sec. 3.1.5), FP32, for sm_103a.
//
// The same u^n as the direct kernel, from a factorisation of the quadrature
// sum.  For node j = (i, k) the tensor Gauss-Hermite points of Eq. (e31) are
// X_p x Y_q: their x coordinate does not depend on q nor their y coordinate
// on p, because the drift and sigma are evaluated at the node.  The
// zero-twist bicubic Hermite interpolant of Eq. (Lag11) is a sum over the
// four corners of a cell of (value, h u_x, h u_y) times products of 1D
// Hermite functions, so
//
//   sum_{p,q} w_p w_q Itilde(X_p, Y_q)
//     = sum_{c,r} u_{c,r} phi_c Phi_r + h u_x(c,r) psi_c Phi_r + h u_y(c,r) phi_c Psi_r
//
// with 1D weights phi_c = sum_p w_p H(value basis of node c at X_p), psi_c
// the same with the slope basis, and Phi_r, Psi_r along y.  The nodes with
// a non-zero weight lie in a W x W window: point p falls in cell
// c_0 + m_p + beta_p, where m_p = floor(g_p - g_0) is a plan constant and
// beta_p is 0 or 1, so W = m_{Q-1} + 3.
//
// Exits (Eq. (e24)): point (p, q) takes the value 1 when X_p or Y_q is
// outside the closed box.  Dropping such points from the 1D weights keeps
// the sum separable:
//
//   u^n_j = u_j + sum_{c,r} [(u_{c,r} - u_j) phi_c Phi_r + ...]      (masked weights)
//             + (1 - u_j) (E_x + E_y - E_x E_y),
//
// where E_x and E_y are the weights of the dropped x- and y-points.  The
// exit term is exactly 0 for a node whose points all stay inside, and the
// window part is in the increment form u_j + sum w (Itilde - u_j), so that
// rounding scales with the per-step change.  Every interior node, next to
// a face or not, takes the same branch-free path.
//
// Per CTA (32 x ty output nodes): stage u^{n+1} over the tile plus halo
// with cp.async, form the scaled PCHIP slopes of Eq. (e300) into one 16-byte
// record {u, h u_x, h u_y, 0} per staged node, then per node: the x and y
// weights as f32x2 pairs (both axes at once), the W x W record window, and
// the exit term.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {


// Adds the contributions (v0, v1, v2) of one point to slots m, m+1, m+2 of
// the value weights PH and (s0, s1, s2) to the slope weights PS.  m is the
// same for every thread (a plan constant), so the switch is a uniform
// branch and the weight arrays stay in registers.
template <int W, int M>
struct Scatter {
  __device__ __forceinline__ static void run(int m, float2* PH, float2* PS, float2 v0, float2 v1,
                                             float2 v2, float2 s0, float2 s1, float2 s2) {
    if (m == M) {
      PH[M] = add2(PH[M], v0);
      PH[M + 1] = add2(PH[M + 1], v1);
      PH[M + 2] = add2(PH[M + 2], v2);
      PS[M] = add2(PS[M], s0);
      PS[M + 1] = add2(PS[M + 1], s1);
      PS[M + 2] = add2(PS[M + 2], s2);
    } else {
      Scatter<W, M + 1>::run(m, PH, PS, v0, v1, v2, s0, s1, s2);
    }
  }
};
template <int W>
struct Scatter<W, W - 2> {
  __device__ __forceinline__ static void run(int, float2*, float2*, float2, float2, float2, float2,
                                             float2, float2) {}
};

// MINB: CTAs of 256 threads per SM the register budget is sized for
// (3 -> 80 registers, 2 -> 128; variant 0 and 1 of the plan).
// MF: several fields per launch (blockIdx.z), for Algorithm 1.
template <int Q, int W, int MINB, bool MF>
__global__ void __launch_bounds__(FK_THREADS, MINB) k_step2dm(const Step2D<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lx = a.lx, ly = a.ly, lp = a.lyr;  // staged extent; lp: odd row pitch
  // per point q: {gx, gy, -m, -m}, {w, w, 0, 0}; then {1, 1, 3, 3}, {-2, -2, 0, 0}
  float4* QC = reinterpret_cast<float4*>(smem);
  float4* Rec = QC + 2 * FK_MAXQ_2D + 2;
  float* U = reinterpret_cast<float*>(Rec + ly * lp);
  const int tid = threadIdx.x;
  if (tid < Q) {
    QC[2 * tid] = make_float4(a.gx[tid], a.gy[tid], -a.wmf[tid], -a.wmf[tid]);
    QC[2 * tid + 1] = make_float4(a.w[tid], a.w[tid], 0.f, 0.f);
  }
  if (tid == 0) {
    QC[2 * FK_MAXQ_2D] = make_float4(1.f, 1.f, 3.f, 3.f);
    QC[2 * FK_MAXQ_2D + 1] = make_float4(-2.f, -2.f, 0.f, 0.f);
  }
  const int i0 = 1 + blockIdx.x * 32, k0 = 1 + blockIdx.y * a.ty;
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;  // global node of staged (0, 0)

  masked_stage<MF>(a, Rec, U, gi0, gk0);

  // 3. one output node per thread and pass: column i0 + lane, row k0 + warp + 8 m
  const int lane = tid & 31, warp = tid >> 5;
  const int i = i0 + lane;
  if (i > a.nx - 2) return;
  const int li = i - gi0;
  // column factors of the cellular drift: A sin(pi x) + e1 sin(2 pi x) and
  // A cos(pi x) + e2 cos(2 pi x) (constant drift: 1, the row factor is the drift)
  float fcx = 1.f, fcy = 1.f;
  if (a.family == FK_CELLULAR_FLOW) {
    const float* ct = a.col_tab + 4 * (int64_t)i;
    fcx = a.A * ct[0] + a.e1 * ct[1];
    fcy = a.A * ct[2] + a.e2 * ct[3];
  }
  unsigned bad = 0;
#pragma unroll 1
  for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
    const int k = k0 + ty;
    if (k > a.ny - 2) break;
    const int lk = k - gk0;
    const float uj = U[lk * lp + li];
    float dx, dy;
    if (a.family == FK_CELLULAR_FLOW) {
      const float* rt = a.row_tab + 2 * (int64_t)k;
      dx = a.kx * rt[0] * fcx;
      dy = a.ky * rt[1] * fcy;
    } else {
      dx = a.cdx * fcx;
      dy = a.cdy * fcy;
    }
    // window origin F0: the cell of point 0 on each axis; positions are
    // then taken after it, s = Z + g_q with Z = D - F0, and a point exits
    // when s leaves [LO, HI] (the box in the same coordinates)
    const float fx0 = floorf(dx + a.gx[0]), fy0 = floorf(dy + a.gy[0]);
    int wx = li + (int)fx0, wy = lk + (int)fy0;
    if (wx < 1 || wx + W - 1 > lx - 2 || wy < 1 || wy + W - 1 > ly - 2) {
      bad = 1u;  // halo too small for this drift: flag, read an in-range window
      wx = 1;
      wy = 1;
    }
    const float2 Z = f2(dx - fx0, dy - fy0);
    const float2 LO = f2(-(float)i - fx0, -(float)k - fy0);
    const float2 HI = f2((float)(a.nx - 1 - i) - fx0, (float)(a.ny - 1 - k) - fy0);
    // 1D weights, x in .x and y in .y: PH[s] = (phi_s, Phi_s), PS[s] = (psi_s, Psi_s)
    float2 PH[W], PS[W];
#pragma unroll
    for (int r = 0; r < W; ++r) PH[r] = PS[r] = f2(0.f, 0.f);
    float2 E = f2(0.f, 0.f);
    const float4* qc = QC + opaque_zero();
    const float4 kc0 = qc[2 * FK_MAXQ_2D], kc1 = qc[2 * FK_MAXQ_2D + 1];
    const float2 ONE = f2(kc0.x, kc0.y), THREE = f2(kc0.z, kc0.w), MTWO = f2(kc1.x, kc1.y);
    // (unrolled by two: full unrolling lets the scheduler overlap so many
    // points that the weights no longer fit the register budget)
#pragma unroll 2
    for (int q = 0; q < Q; ++q) {
      const float4 k0q = qc[2 * q], k1q = qc[2 * q + 1];
      const float wq = k1q.x;
      const float2 sq = add2(Z, f2(k0q.x, k0q.y));
      // position within the two cells m_q, m_q + 1 of the window
      const float2 tp = add2(sq, f2(k0q.z, k0q.w));
      const float2 beta = f2(tp.x >= 1.f ? 1.f : 0.f, tp.y >= 1.f ? 1.f : 0.f);
      const float2 t = add2(tp, f2(-beta.x, -beta.y));
      const float2 ex = f2((sq.x < LO.x || sq.x > HI.x) ? wq : 0.f,
                           (sq.y < LO.y || sq.y > HI.y) ? wq : 0.f);
      E = add2(E, ex);
      const float2 wm = add2(f2(k1q.x, k1q.y), f2(-ex.x, -ex.y));  // weight, 0 if the point exits
      // cubic Hermite basis at t, weighted: values (v0, v1), slopes (s0, s1)
      const float2 tt = mul2(t, t);
      const float2 omt = add2(ONE, f2(-t.x, -t.y));
      const float2 v1 = mul2(wm, mul2(tt, fma2(MTWO, t, THREE)));
      const float2 v0 = add2(wm, f2(-v1.x, -v1.y));
      const float2 wt = mul2(wm, t);
      const float2 s0 = mul2(mul2(wt, omt), omt);
      const float2 s1 = mul2(mul2(wt, t), f2(-omt.x, -omt.y));
      // beta = 1 moves the pair one node up: slots (m, m+1, m+2) get
      // ((1-beta) v0, v1 + beta (v0 - v1), beta v1)
      const float2 nb = f2(-beta.x, -beta.y);
      const float2 b0 = fma2(nb, v0, v0), b2 = mul2(beta, v1);
      const float2 b1 = fma2(beta, add2(v0, f2(-v1.x, -v1.y)), v1);
      const float2 c0 = fma2(nb, s0, s0), c2 = mul2(beta, s1);
      const float2 c1 = fma2(beta, add2(s0, f2(-s1.x, -s1.y)), s1);
      Scatter<W, 0>::run(a.wm[q], PH, PS, b0, b1, b2, c0, c1, c2);
    }
    // W x W record window, row by row:
    //   (Ae_r, Ax_r) = sum_c (phi_c, psi_c) * (u - u_j, h u_x),  B_r = sum_c phi_c h u_y,
    //   acc += Phi_r (Ae_r + Ax_r) + Psi_r B_r
    float2 XP[W];  // (phi_c, psi_c)
    float PY[W], SY[W];  // Phi_r, Psi_r
#pragma unroll
    for (int c = 0; c < W; ++c) {
      XP[c] = f2(PH[c].x, PS[c].x);
      PY[c] = PH[c].y;
      SY[c] = PS[c].y;
    }
    const float4* win = Rec + (wy * lp + wx);
    const float2 ujz = f2(-uj, 0.f);
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const float4* row = win + r * lp;
      float2 AE = f2(0.f, 0.f);
      float B = 0.f;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float4 v = row[c];
        AE = fma2(XP[c], add2(f2(v.x, v.y), ujz), AE);
        B = fmaf(XP[c].x, v.z, B);
      }
      acc = fmaf(PY[r], AE.x + AE.y, fmaf(SY[r], B, acc));
    }
    const float ext = (1.f - uj) * (E.x + E.y - E.x * E.y);
    const float un = uj + (acc + ext);
    const int64_t j = (int64_t)k * a.nx + i;
    field_out<MF>(a)[j] = un;
    if (a.snap) a.snap[j] = un;
    write_adjacent_boundary<MF>(a, i, k);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// Several fields run the 3-CTA/SM register budget whatever the variant.
template <int Q, int W, int MINB>
cudaError_t launch_m(const Step2D<float>& a, cudaStream_t s) {
  const size_t smem = fk_step2dm_smem(a.ly, a.lyr);
  const int nf = a.ncols > 1 ? a.ncols : 1;
  dim3 grid((a.nx - 2 + 31) / 32, (a.ny - 2 + a.ty - 1) / a.ty, nf);
  if (nf > 1)
    k_step2dm<Q, W, 3, true><<<grid, FK_THREADS, smem, s>>>(a);
  else
    k_step2dm<Q, W, MINB, false><<<grid, FK_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int Q, int W>
cudaError_t attr_m() {
  const int big = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_step2dm<Q, W, 3, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step2dm<Q, W, 2, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step2dm<Q, W, 3, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

}  // namespace

size_t fk_step2dm_smem(int ly, int lp) {
  return (size_t)(2 * FK_MAXQ_2D + 2) * 16 + (size_t)ly * lp * (16 + 4);
}

bool fk_masked_available(int q, int w) {
#define FK_M(QQ, WW) \
  if (q == QQ && w == WW) return true;
  FK_MASKED_LIST(FK_M)
#undef FK_M
  return false;
}

cudaError_t fk_launch_step2dm(const Step2D<float>& a, int q, cudaStream_t s) {
#define FK_M(QQ, WW)                                                           \
  if (q == QQ && a.win == WW)                                                  \
    return a.variant == 1 ? launch_m<QQ, WW, 2>(a, s) : launch_m<QQ, WW, 3>(a, s);
  FK_MASKED_LIST(FK_M)
#undef FK_M
  return cudaErrorInvalidValue;
}

cudaError_t fk_prepare_masked_kernels(int q) {
#define FK_M(QQ, WW)                   \
  if (q == QQ) {                       \
    cudaError_t e = attr_m<QQ, WW>();  \
    if (e != cudaSuccess) return e;    \
  }
  FK_MASKED_LIST(FK_M)
#undef FK_M
  return cudaSuccess;
}
