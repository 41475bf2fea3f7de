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
// a non-zero weight lie in a W x W window: point q falls in cell
// c_0 + m_q + beta_q, where m_q = floor(g_q - g_0) is a plan constant (one
// of the patterns fk_mpat lists) and beta_q is 0 or 1, so W = m_{Q-1} + 3.
// The kernel is compiled for every pattern of its (Q, W) and takes the
// plan's with one uniform branch, so each point's weights land in fixed
// registers.
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
// rounding scales with the per-step change.  Rows of nodes whose points
// cannot leave the box (tiles at least a halo away from the x faces, rows
// at least a halo away from the y faces) skip the exit tests.
//
// Per CTA (32 x ty output nodes): stage u^{n+1} over the tile plus halo
// with cp.async, form the scaled PCHIP slopes of Eq. (e300) and store, for
// every staged node c, the pair records {u_c, u_{c+1}, h u_x(c),
// h u_x(c+1)} and {h u_y(c), h u_y(c+1)}; then per node: the x and y
// weights as f32x2 pairs (both axes at once), and the window read as pairs
// of columns, so that each f32x2 multiply-add covers two nodes of the
// window.  (Tiled TMA copies cannot stage these fields: a row of 2^k + 1
// FP32 values is not a multiple of 16 bytes long.)
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fk_device.cuh"
#include "fk_internal.h"

namespace {

// Pair records of the staged tile (lx x ly nodes, row pitch lx): P[r][c] =
// {u_c, u_{c+1}, h u_x(c), h u_x(c+1)} and Y[r][c] = {h u_y(c), h u_y(c+1)}
// for staged columns c = 1 .. lx-3 and rows r = 1 .. ly-2; U holds u^{n+1}
// itself (zero outside the mesh), from field = u^{n+1}.  Ends with the
// records visible to the whole CTA.  (In the persistent march the copies
// follow a gpu-scope acquire of the neighbours' step counts and a CTA
// barrier, which is what makes the neighbours' stores visible to them.)
__device__ __forceinline__ void stage_pairs(const Step2D<float>& a, const float* field, float* U,
                                            float4* P, float2* Y, int gi0, int gk0) {
  const int lx = a.lx, ly = a.ly;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // 1. u^{n+1} over the tile and halo: rows by warp, columns by lane, so
  // global reads are coalesced and shared-memory writes consecutive.  A lane
  // holds columns lane and lane + 32 (more only for halos over 14 nodes);
  // reads outside the mesh are clamped to a mesh node and copy 0 bytes (zero
  // fill)
  {
    const uint32_t sU = (uint32_t)__cvta_generic_to_shared(U);
    const int c1 = lane + 32;
    const int g0 = gi0 + lane, g1 = gi0 + c1;
    const bool x0 = (unsigned)g0 < (unsigned)a.nx, x1 = c1 < lx && (unsigned)g1 < (unsigned)a.nx;
    const int cx0 = min(max(g0, 0), a.nx - 1), cx1 = min(max(g1, 0), a.nx - 1);
    const float* base = field;
#pragma unroll 1
    for (int r = warp; r < ly; r += FK_THREADS / 32) {
      const int gk = gk0 + r;
      const bool rowin = (unsigned)gk < (unsigned)a.ny;
      const float* src = base + (int64_t)min(max(gk, 0), a.ny - 1) * a.nx;
      const uint32_t drow = sU + (uint32_t)(r * lx) * 4u;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(drow + 4u * lane),
                   "l"(src + cx0), "r"(rowin && x0 ? 4 : 0));
      if (c1 < lx)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(drow + 4u * c1),
                     "l"(src + cx1), "r"(rowin && x1 ? 4 : 0));
      for (int c = lane + 64; c < lx; c += 32) {  // wide halos only
        const int g = gi0 + c;
        const bool in = rowin && (unsigned)g < (unsigned)a.nx;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(drow + 4u * c),
                     "l"(src + min(max(g, 0), a.nx - 1)), "r"(in ? 4 : 0));
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
  }
  // 2. vertical sweeps: warp group g takes staged columns 1 + 31 g + lane
  // (lane 31 lends its values to lane 30 and stores nothing) over one
  // segment of rows, carrying u of the rows above and below in registers;
  // the partner column's values come by shuffle.  The end rule stated after
  // Eq. (e300) gives node 0 the slope of node 1 and node n-1 that of node
  // n-2 (the harmonic mean is symmetric): an end column takes its
  // x-differences one column inwards, and the end rows copy the y-slopes of
  // their neighbour row afterwards.  Nodes outside the mesh get finite
  // values from the zero fill; they only ever carry weight 0.
  {
    const int groups = (lx - 3 + 30) / 31;
    const int segs = (FK_THREADS / 32) / groups;
    const int g = warp % groups, seg = warp / groups;
    if (seg < segs) {
      const int c = 1 + 31 * g + lane;
      const bool have = c <= lx - 2;  // slopes exist for staged columns 1 .. lx-2
      const bool emit = lane < 31 && c <= lx - 3;
      const int hr = ly - 2;
      const int len = (hr + segs - 1) / segs;
      const int r0 = 1 + seg * len, r1 = min(r0 + len, hr + 1);
      const int gi = gi0 + c;
      const int ax = c + (gi == 0) - (gi == a.nx - 1);
      const int cc = have ? c : 1, axc = have ? ax : 1;  // idle lanes read in range
      const float* col = U + cc;
      const float* colx = U + axc;
      float up = r0 <= hr ? col[(r0 - 1) * lx] : 0.f, uc = r0 <= hr ? col[r0 * lx] : 0.f;
      for (int r = r0; r < r1; ++r) {
        const float un = col[(r + 1) * lx];
        const float* rx = colx + r * lx;
        const float X = pchip_rcp(rx[0] - rx[-1], rx[1] - rx[0]);
        const float Yv = pchip_rcp(uc - up, un - uc);
        const float u1 = __shfl_down_sync(0xffffffffu, uc, 1);
        const float X1 = __shfl_down_sync(0xffffffffu, X, 1);
        const float Y1 = __shfl_down_sync(0xffffffffu, Yv, 1);
        if (emit) {
          P[r * lx + c] = make_float4(uc, u1, X, X1);
          Y[r * lx + c] = make_float2(Yv, Y1);
        }
        up = uc;
        uc = un;
      }
    }
    __syncthreads();
    // y end rule: staged rows of mesh rows 0 and ny-1 take their neighbour's y-slopes
    const int rb = -gk0, rt = a.ny - 1 - gk0;
    const bool fb = rb >= 1 && rb <= ly - 3, ft = rt >= 2 && rt <= ly - 2;
    if (fb || ft) {
      for (int e = tid; e < lx - 3; e += FK_THREADS) {
        if (fb) Y[rb * lx + 1 + e] = Y[(rb + 1) * lx + 1 + e];
        if (ft) Y[rt * lx + 1 + e] = Y[(rt - 1) * lx + 1 + e];
      }
      __syncthreads();
    }
  }
}

// The 1D weights of points q .. Q-1 of pattern K of (Q, W), x in .x and y
// in .y: PH[s] += (phi_s, Phi_s), PS[s] += (psi_s, Psi_s).  qc[q] = {G_x,
// G_y, w_q, w_q} with G = g_q - m_q.  Z: the drift after the window
// origin, so that point q sits at Z + g_q = Z + G + m_q.  With EXIT, a point outside [LO, HI] (positions
// after the window origin) is dropped and its weight added to E.
// The first point of pattern K of (Q, W) whose cell pair touches window
// slot s (point q touches slots m_q .. m_q + 2), or Q if none does.
__host__ __device__ constexpr int first_point(int Q, int W, int K, int s) {
  for (int q = 0; q < Q; ++q)
    if (fk_mpat(Q, W, K, q) <= s && s <= fk_mpat(Q, W, K, q) + 2) return q;
  return Q;
}

// a * b + c, or a * b where point q is the first to reach the slot
template <bool FIRST>
__device__ __forceinline__ float2 acc2(float2 a, float2 b, float2 c) {
  if constexpr (FIRST) return mul2(a, b);
  else return fma2(a, b, c);
}

template <int Q, int W, int K, bool EXIT, int q>
struct PointWeights {
  template <int S>
  __device__ __forceinline__ static void run(const float4* qc, float2 Z, float2 LO, float2 HI,
                                             float2 (&PH)[S], float2 (&PS)[S], float2& E) {
    if constexpr (q < Q) {
      constexpr int M = fk_mpat(Q, W, K, q);
      static_assert(M >= 0 && M + 2 < S, "pattern slot outside the window");
      const float4 c0 = qc[q];
      const float2 one = f2(1.f, 1.f);
      const float2 tp = add2(Z, f2(c0.x, c0.y));  // in [0, 2): cells M and M + 1, up to rounding
      float2 w1 = f2(c0.z, c0.w);
      if constexpr (EXIT) {
        const float2 sq = add2(tp, f2((float)M, (float)M));
        const float2 ex = f2((sq.x < LO.x || sq.x > HI.x) ? w1.x : 0.f,
                             (sq.y < LO.y || sq.y > HI.y) ? w1.y : 0.f);
        E = add2(E, ex);
        w1 = add2(w1, f2(-ex.x, -ex.y));  // weight, 0 if the point exits
      }
      // (tp may round a hair outside [0, 2) at a cell face: the cubic is
      // continuous there, so the compare only has to pick one of the cells)
      const float2 beta = f2(tp.x >= 1.f ? 1.f : 0.f, tp.y >= 1.f ? 1.f : 0.f);
      const float2 t = add2(tp, f2(-beta.x, -beta.y));
      const float2 nb = add2(one, f2(-beta.x, -beta.y));
      // cubic Hermite basis at t, weighted: values v0 = w h00, v1 = w h01,
      // slopes s0 = w h10, s1 = w h11.  h01 = t^2 (3 - 2t) is formed before
      // the weight is applied: 3 - 2t is exact, while a rounded 3 w would
      // shift the same sliver of weight from node to node at every node and
      // step, a bias that adds up over a march.
      const float2 tt = mul2(t, t);
      const float2 om = add2(t, f2(-1.f, -1.f));
      const float2 v1 = mul2(w1, mul2(tt, fma2(f2(-2.f, -2.f), t, f2(3.f, 3.f))));
      const float2 v0 = add2(w1, f2(-v1.x, -v1.y));
      const float2 wto = mul2(mul2(w1, t), om);
      const float2 s0 = mul2(wto, om);
      const float2 s1 = mul2(wto, t);
      // beta = 1 moves the pair one node up: slots (M, M+1, M+2) get
      // ((1-beta) v0, beta v0 + (1-beta) v1, beta v1)
      // (a slot's first contribution is a product: no zero fill needed)
      constexpr bool F0 = first_point(Q, W, K, M) == q, F1 = first_point(Q, W, K, M + 1) == q,
                     F2 = first_point(Q, W, K, M + 2) == q;
      PH[M] = acc2<F0>(nb, v0, PH[M]);
      PH[M + 1] = fma2(beta, v0, acc2<F1>(nb, v1, PH[M + 1]));
      PH[M + 2] = acc2<F2>(beta, v1, PH[M + 2]);
      PS[M] = acc2<F0>(nb, s0, PS[M]);
      PS[M + 1] = fma2(beta, s0, acc2<F1>(nb, s1, PS[M + 1]));
      PS[M + 2] = acc2<F2>(beta, s1, PS[M + 2]);
      PointWeights<Q, W, K, EXIT, q + 1>::run(qc, Z, LO, HI, PH, PS, E);
    }
  }
};

// The tile geometry a node body needs: staged tile size, the staged node
// (0, 0) as a global node, and the shared-memory tables.
struct MaskedTileRefs {
  const float4* QC;
  const float4* P;
  const float2* Yr;
  const float* U;
  int lx, ly, gi0, gk0;
};

// What one output node carries from its 1D weights to the window sums: the
// weights PH[s] = (phi_s, Phi_s), PS[s] = (psi_s, Psi_s) over slots s <
// 2 NP (the padding slot of an odd W is 0), the dropped exit weights E,
// u_j, and the window origin (wx, wy) in staged coordinates.
template <int W>
struct MaskedNode {
  static constexpr int NP = (W + 1) / 2;  // column pairs of the window
  float2 PH[2 * NP], PS[2 * NP];
  float2 E;
  float uj;
  int wx, wy;
};

// The 1D weights of node (i, k) for pattern K of (Q, W).
template <int Q, int W, int K, bool EXIT>
__device__ __forceinline__ void masked_weights(const Step2D<float>& a, const MaskedTileRefs& t,
                                               int i, int k, float fcx, float fcy,
                                               MaskedNode<W>& n, unsigned& bad) {
  constexpr int NP = MaskedNode<W>::NP;
  const int lx = t.lx, ly = t.ly;
  const int li = i - t.gi0, lk = k - t.gk0;
  n.uj = t.U[lk * lx + li];
  float dx, dy;
  if (a.family == FK_CELLULAR_FLOW) {
    const float* rt = a.row_tab + 2 * (int64_t)k;
    dx = a.kx * rt[0] * fcx;
    dy = a.ky * rt[1] * fcy;
  } else {
    dx = a.cdx * fcx;
    dy = a.cdy * fcy;
  }
  // window origin F0: the cell of point 0 on each axis; positions after
  // it are Z + g_q with Z = D - F0 (the points keep the rule's symmetric
  // offsets g_q, so FP32 rounding of the offsets cannot add up to a drift),
  // and a point exits when it leaves [LO, HI] (the box in the same
  // coordinates)
  const float fx0 = floorf(dx + a.gx[0]), fy0 = floorf(dy + a.gy[0]);
  n.wx = li + (int)fx0;
  n.wy = lk + (int)fy0;
  if (n.wx < 1 || n.wx + 2 * NP - 1 > lx - 2 || n.wy < 1 || n.wy + W - 1 > ly - 2) {
    bad = 1u;  // halo too small for this drift: flag, read an in-range window
    n.wx = 1;
    n.wy = 1;
  }
  const float2 Z = f2(dx - fx0, dy - fy0);
  float2 LO = f2(0.f, 0.f), HI = f2(0.f, 0.f);
  if constexpr (EXIT) {
    LO = f2(-(float)i - fx0, -(float)k - fy0);
    HI = f2((float)(a.nx - 1 - i) - fx0, (float)(a.ny - 1 - k) - fy0);
  }
  // (slots 0 .. W-1 all receive a first contribution; the padding slot of
  // an odd W stays 0)
#pragma unroll
  for (int r = W; r < 2 * NP; ++r) n.PH[r] = n.PS[r] = f2(0.f, 0.f);
  n.E = f2(0.f, 0.f);
  PointWeights<Q, W, K, EXIT, 0>::run(t.QC + opaque_zero(), Z, LO, HI, n.PH, n.PS, n.E);
}

// The W x W record window of one node, row by row, two columns per f32x2
// operation:
//   (AE_r, AX_r) = sum_c (phi_c (u - u_j), psi_c h u_x),  B_r = sum_c phi_c h u_y,
//   acc += Phi_r (AE_r + AX_r) + Psi_r B_r
// (An odd W reads its last column as a whole pair whose second weight is
// 0: reading it as three scalars instead halves its bytes but adds an
// instruction per row, and the kernel is issue-bound: a GB300 ran the
// 1025 x 513 march 0.5-5 % slower that way.)
template <int W>
__device__ __forceinline__ float masked_window(const MaskedTileRefs& t, const MaskedNode<W>& n) {
  constexpr int NP = MaskedNode<W>::NP;
  const int lx = t.lx;
  float2 XP[NP], XS[NP];  // (phi_c, phi_c+1), (psi_c, psi_c+1), c = 2 j
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    XP[j] = f2(n.PH[2 * j].x, n.PH[2 * j + 1].x);
    XS[j] = f2(n.PS[2 * j].x, n.PS[2 * j + 1].x);
  }
  const float4* pwin = t.P + (n.wy * lx + n.wx);
  const float2* ywin = t.Yr + (n.wy * lx + n.wx);
  const float2 nuj = f2(-n.uj, -n.uj);
  float acc = 0.f;
#pragma unroll
  for (int r = 0; r < W; ++r) {
    const float4* pr = pwin + r * lx;
    const float2* yr = ywin + r * lx;
    float2 AE, AX, B;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float4 p = pr[2 * j];
      const float2 y = yr[2 * j];
      const float2 du = add2(f2(p.x, p.y), nuj);
      if (j == 0) {
        AE = mul2(XP[0], du);
        AX = mul2(XS[0], f2(p.z, p.w));
        B = mul2(XP[0], y);
      } else {
        AE = fma2(XP[j], du, AE);
        AX = fma2(XS[j], f2(p.z, p.w), AX);
        B = fma2(XP[j], y, B);
      }
    }
    const float2 T = add2(AE, AX);
    acc = fmaf(n.PH[r].y, T.x + T.y, fmaf(n.PS[r].y, B.x + B.y, acc));
  }
  return acc;
}

// The exit term of node n: (1 - u_j) (E_x + E_y - E_x E_y).
template <bool EXIT, int W>
__device__ __forceinline__ float masked_exit(const MaskedNode<W>& n) {
  return EXIT ? (1.f - n.uj) * (n.E.x + n.E.y - n.E.x * n.E.y) : 0.f;
}

// u^n of node (i, k) from its window sum and exit term: the increment
// form, the store and the boundary nodes next to it.
template <int W>
__device__ __forceinline__ void masked_store(const Step2D<float>& a, float* u_out, int i, int k,
                                             const MaskedNode<W>& n, float acc, float ext) {
  const float un = n.uj + (acc + ext);
  const int64_t j = (int64_t)k * a.nx + i;
  u_out[j] = un;
  if (a.snap) a.snap[j] = un;
  boundary_ones(u_out, a.snap, a.nx, a.ny, i, k);
}

// One output node (i, k) of pattern K of (Q, W): its 1D weights, the W x W
// record window and the store.  Compiled per pattern and exit flag, so the
// weights sit in fixed registers from their first contribution to the last
// read, with no branch join in between.
template <int Q, int W, int K, bool EXIT>
__device__ __forceinline__ void masked_node(const Step2D<float>& a, const MaskedTileRefs& t,
                                            float* u_out, int i, int k, float fcx, float fcy,
                                            unsigned& bad) {
  MaskedNode<W> n;
  masked_weights<Q, W, K, EXIT>(a, t, i, k, fcx, fcy, n, bad);
  const float ext = masked_exit<EXIT>(n);
  masked_store<W>(a, u_out, i, k, n, masked_window<W>(t, n), ext);
}

// Two nodes of one column, A = (i, k) and B = (i, k + 1), from one read of
// the window rows they share (odd W).  B's window sits dy = wy_B - wy_A
// rows below A's (1 for a smooth drift, 0 or 2 where floor(drift) steps
// between the rows) and dx = wx_B - wx_A columns to the side (0, or +-1
// where it steps).  The union of the two windows is then W + 1 rows (W + 2
// when dy = 2) of the same 2 NP = W + 1 columns from ox = min(wx_A,
// wx_B): each node's W columns start at offset 0 or 1 in it, so its weights
// move up one slot when the offset is 1.  Rows read once serve both nodes:
// (W + 1) NP pair records for two nodes instead of 2 W NP.  Slots outside a
// node's window carry weight exactly 0, so each node's sum is its own
// window's, up to the grouping of columns into pairs.  Other offsets (not
// met by a drift that changes by less than a cell between rows) run the
// two windows one after the other.
template <int W>
__device__ __forceinline__ void masked_pair_window(const MaskedTileRefs& t,
                                                   const MaskedNode<W>& A,
                                                   const MaskedNode<W>& B, float& acc_a,
                                                   float& acc_b) {
  constexpr int NP = MaskedNode<W>::NP;
  static_assert(2 * NP == W + 1, "pairs of nodes need an odd window width");
  const int lx = t.lx, ly = t.ly;
  const int ox = min(A.wx, B.wx);
  const bool sa = A.wx != ox, sb = B.wx != ox;  // window starts one column into the union
  const int dy = B.wy - A.wy;                     // 0, 1 or 2
  // x weights on the union's column pairs (2 j, 2 j + 1)
  float2 XPA[NP], XSA[NP], XPB[NP], XSB[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float pa0 = j > 0 ? A.PH[2 * j - 1].x : 0.f, sa0 = j > 0 ? A.PS[2 * j - 1].x : 0.f;
    const float pb0 = j > 0 ? B.PH[2 * j - 1].x : 0.f, sb0 = j > 0 ? B.PS[2 * j - 1].x : 0.f;
    XPA[j] = sa ? f2(pa0, A.PH[2 * j].x) : f2(A.PH[2 * j].x, A.PH[2 * j + 1].x);
    XSA[j] = sa ? f2(sa0, A.PS[2 * j].x) : f2(A.PS[2 * j].x, A.PS[2 * j + 1].x);
    XPB[j] = sb ? f2(pb0, B.PH[2 * j].x) : f2(B.PH[2 * j].x, B.PH[2 * j + 1].x);
    XSB[j] = sb ? f2(sb0, B.PS[2 * j].x) : f2(B.PS[2 * j].x, B.PS[2 * j + 1].x);
  }
  // B's row weights on union rows 0 .. W (slot r - dy; slot W is the padding slot, 0)
  float PHB[W + 1], PSB[W + 1];
#pragma unroll
  for (int r = 0; r <= W; ++r) {
    const float ph1 = r >= 1 ? B.PH[r - 1].y : 0.f, ps1 = r >= 1 ? B.PS[r - 1].y : 0.f;
    const float ph2 = r >= 2 ? B.PH[r - 2].y : 0.f, ps2 = r >= 2 ? B.PS[r - 2].y : 0.f;
    PHB[r] = dy == 0 ? B.PH[r].y : (dy == 1 ? ph1 : ph2);
    PSB[r] = dy == 0 ? B.PS[r].y : (dy == 1 ? ps1 : ps2);
  }
  const float4* pwin = t.P + (A.wy * lx + ox);
  const float2* ywin = t.Yr + (A.wy * lx + ox);
  // union row W is B's last row when dy >= 1; when dy = 0 it lies past both
  // windows (weight 0) and may lie past the records: read an in-range row
  const int rw = min(W, ly - 2 - A.wy);
  const float2 nua = f2(-A.uj, -A.uj), nub = f2(-B.uj, -B.uj);
  float accA = 0.f, accB = 0.f;
#pragma unroll
  for (int r = 0; r <= W; ++r) {
    const int ro = r < W ? r : rw;
    const float4* pr = pwin + ro * lx;
    const float2* yr = ywin + ro * lx;
    float2 Ta, Ba, Tb, Bb;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float4 p = pr[2 * j];
      const float2 y = yr[2 * j];
      const float2 u = f2(p.x, p.y), ux = f2(p.z, p.w);
      if (r < W) {
        const float2 du = add2(u, nua);
        if (j == 0) {
          Ta = fma2(XSA[0], ux, mul2(XPA[0], du));
          Ba = mul2(XPA[0], y);
        } else {
          Ta = fma2(XSA[j], ux, fma2(XPA[j], du, Ta));
          Ba = fma2(XPA[j], y, Ba);
        }
      }
      const float2 dub = add2(u, nub);
      if (j == 0) {
        Tb = fma2(XSB[0], ux, mul2(XPB[0], dub));
        Bb = mul2(XPB[0], y);
      } else {
        Tb = fma2(XSB[j], ux, fma2(XPB[j], dub, Tb));
        Bb = fma2(XPB[j], y, Bb);
      }
    }
    if (r < W) accA = fmaf(A.PH[r].y, Ta.x + Ta.y, fmaf(A.PS[r].y, Ba.x + Ba.y, accA));
    accB = fmaf(PHB[r], Tb.x + Tb.y, fmaf(PSB[r], Bb.x + Bb.y, accB));
  }
  if (dy == 2) {  // B's last row, union row W + 1
    const float4* pr = pwin + (W + 1) * lx;
    const float2* yr = ywin + (W + 1) * lx;
    float2 Tb, Bb;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float4 p = pr[2 * j];
      const float2 y = yr[2 * j];
      const float2 dub = add2(f2(p.x, p.y), nub);
      if (j == 0) {
        Tb = fma2(XSB[0], f2(p.z, p.w), mul2(XPB[0], dub));
        Bb = mul2(XPB[0], y);
      } else {
        Tb = fma2(XSB[j], f2(p.z, p.w), fma2(XPB[j], dub, Tb));
        Bb = fma2(XPB[j], y, Bb);
      }
    }
    accB = fmaf(B.PH[W - 1].y, Tb.x + Tb.y, fmaf(B.PS[W - 1].y, Bb.x + Bb.y, accB));
  }
  acc_a = accA;
  acc_b = accB;
}

// Nodes (i, k) and (i, k + 1) of pattern K of (Q, W); B = (i, k + 1) is
// stored only when store_b (it may be the boundary row ny - 1, whose
// window the halo still covers: it lies in the tile).
template <int Q, int W, int K, bool EXIT>
__device__ __forceinline__ void masked_pair(const Step2D<float>& a, const MaskedTileRefs& t,
                                            float* u_out, int i, int k, bool store_b, float fcx,
                                            float fcy, unsigned& bad) {
  MaskedNode<W> A, B;
  masked_weights<Q, W, K, EXIT>(a, t, i, k, fcx, fcy, A, bad);
  masked_weights<Q, W, K, EXIT>(a, t, i, k + 1, fcx, fcy, B, bad);
  // (the exit terms first: the dropped weights need not stay live across the window)
  const float ext_a = masked_exit<EXIT>(A), ext_b = masked_exit<EXIT>(B);
  float acc_a, acc_b;
  const int dx = B.wx - A.wx, dy = B.wy - A.wy;
  if (dx >= -1 && dx <= 1 && dy >= 0 && dy <= 2) {
    masked_pair_window<W>(t, A, B, acc_a, acc_b);
  } else {
    acc_a = masked_window<W>(t, A);
    acc_b = masked_window<W>(t, B);
  }
  masked_store<W>(a, u_out, i, k, A, acc_a, ext_a);
  if (store_b) masked_store<W>(a, u_out, i, k + 1, B, acc_b, ext_b);
}

// The rows of one tile column (one output node per thread and pass: column
// i, rows k0 + warp + 8 m; PAIR: two nodes per thread and pass, rows
// k0 + 2 warp + 16 m and the row after it, the tile height being even)
// with pattern K; a row whose points can leave the box takes the exit
// tests.
template <int Q, int W, int K, bool PAIR>
__device__ __forceinline__ void masked_rows(const Step2D<float>& a, const MaskedTileRefs& t,
                                            float* u_out, int i, int k0, bool xsafe, float fcx,
                                            float fcy, unsigned& bad) {
  const int warp = threadIdx.x >> 5;
  if constexpr (PAIR) {
#pragma unroll 1
    for (int ty = 2 * warp; ty < a.ty; ty += 2 * (FK_THREADS / 32)) {
      const int k = k0 + ty;
      if (k > a.ny - 2) break;
      const bool store_b = k + 1 <= a.ny - 2;
      if (!(xsafe && k - a.hy >= 0 && k + 1 + a.hy <= a.ny - 1))
        masked_pair<Q, W, K, true>(a, t, u_out, i, k, store_b, fcx, fcy, bad);
      else
        masked_pair<Q, W, K, false>(a, t, u_out, i, k, store_b, fcx, fcy, bad);
    }
  } else {
#pragma unroll 1
    for (int ty = warp; ty < a.ty; ty += FK_THREADS / 32) {
      const int k = k0 + ty;
      if (k > a.ny - 2) break;
      if (!(xsafe && k - a.hy >= 0 && k + a.hy <= a.ny - 1))
        masked_node<Q, W, K, true>(a, t, u_out, i, k, fcx, fcy, bad);
      else
        masked_node<Q, W, K, false>(a, t, u_out, i, k, fcx, fcy, bad);
    }
  }
}

// The plan's pattern `pat` of (Q, W), taken from K upwards: one uniform
// branch per tile, ahead of the row loop.
template <int Q, int W, int K, bool PAIR>
__device__ __forceinline__ void masked_rows_of(int pat, const Step2D<float>& a,
                                               const MaskedTileRefs& t, float* u_out, int i,
                                               int k0, bool xsafe, float fcx, float fcy,
                                               unsigned& bad) {
  if constexpr (K < fk_npat(Q, W)) {
    if (pat == K)
      masked_rows<Q, W, K, PAIR>(a, t, u_out, i, k0, xsafe, fcx, fcy, bad);
    else
      masked_rows_of<Q, W, K + 1, PAIR>(pat, a, t, u_out, i, k0, xsafe, fcx, fcy, bad);
  }
}

// One tile (bx, by) of one step: u_in -> u_out (and a.snap), with the
// per-step drift factors e1, e2 of the cellular flow.  MF: u_in and u_out
// are the field of blockIdx.z.  PAIR: two nodes of a column per thread
// (odd W, even tile height).  Sets bad when a halo range check fires.
template <int Q, int W, bool MF, bool PAIR>
__device__ __forceinline__ void masked_tile(const Step2D<float>& a, const float* u_in,
                                            float* u_out, float e1, float e2, int bx, int by,
                                            unsigned char* smem, unsigned& bad) {
  const int lx = a.lx, ly = a.ly;
  float4* QC = reinterpret_cast<float4*>(smem);
  float4* P = QC + FK_MAXQ_2D;
  float2* Yr = reinterpret_cast<float2*>(P + ly * lx);
  float* U = reinterpret_cast<float*>(Yr + ly * lx);
  const int tid = threadIdx.x;
  if (tid < Q) QC[tid] = make_float4(a.gmx[tid], a.gmy[tid], a.w[tid], a.w[tid]);
  const int i0 = 1 + bx * 32, k0 = 1 + by * a.ty;
  const int gi0 = i0 - a.hx - 1, gk0 = k0 - a.hy - 1;  // global node of staged (0, 0)

  stage_pairs(a, u_in, U, P, Yr, gi0, gk0);

  // 3. the output nodes: column i0 + lane of the tile, every row
  const int lane = tid & 31;
  const int i = i0 + lane;
  if (i > a.nx - 2) return;  // (no barrier follows in the tile)
  // no point of a node in this tile's columns can leave through an x face
  // (the halo exceeds the reach of every point)
  const bool xsafe = i0 - a.hx >= 0 && i0 + 31 + a.hx <= a.nx - 1;
  // column factors of the cellular drift: A sin(pi x) + e1 sin(2 pi x) and
  // A cos(pi x) + e2 cos(2 pi x) (constant drift: 1, the row factor is the drift)
  float fcx = 1.f, fcy = 1.f;
  if (a.family == FK_CELLULAR_FLOW) {
    const float* ct = a.col_tab + 4 * (int64_t)i;
    fcx = a.A * ct[0] + e1 * ct[1];
    fcy = a.A * ct[2] + e2 * ct[3];
  }
  const MaskedTileRefs t = {QC, P, Yr, U, lx, ly, gi0, gk0};
  masked_rows_of<Q, W, 0, PAIR>(a.mpat, a, t, u_out, i, k0, xsafe, fcx, fcy, bad);
}

// MINB: CTAs of 256 threads per SM the register budget is sized for
// (3 -> 80 registers, 2 -> 128, 4 -> 64; variants 0, 1 and 2 of the plan;
// variant 3 is PAIR with 2).
// MF: several fields per launch (blockIdx.z), for Algorithm 1.
template <int Q, int W, int MINB, bool MF, bool PAIR = false>
__global__ void __launch_bounds__(FK_THREADS, MINB) k_step2dm(const Step2D<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned bad = 0;
  masked_tile<Q, W, MF, PAIR>(a, field_in<MF>(a), field_out<MF>(a), a.e1, a.e2, blockIdx.x,
                              blockIdx.y, smem, bad);
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// The persistent march: steps n_from-1 .. n_to of Scheme 1 in one launch,
// one CTA per tile (all co-resident: a cooperative launch).  A tile starts
// step m once the tiles around it (the 3 x 3 block: its halo is smaller
// than a tile) have finished step m-1, signalled by a per-tile count of
// finished steps (release after the CTA's stores, acquire before staging;
// one lane per neighbour polls, so the wait costs one L2 round trip once
// every neighbour is done).
// No tile is ever more than one step ahead of a neighbour, so two buffers
// suffice: step m writes buf[(steps - m) & 1] while every tile that still
// reads that buffer's previous contents has finished.  Staging of one
// tile overlaps the compute of others, and no step waits for the slowest
// CTA of the grid or for a launch.  A wait is bounded: after 1 s (or 2^24
// polls) the CTA records FK_DEVERR_TIMEOUT and raises the abort word, and
// every CTA leaves at its next wait.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int Q, int W, int MINB, bool PAIR = false>
__global__ void __launch_bounds__(FK_THREADS, MINB) k_march2dm(const Step2D<float> a,
                                                               const MaskedMarch m) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int go;
  const int bx = blockIdx.x, by = blockIdx.y, tx = gridDim.x, tyn = gridDim.y;
  unsigned bad = 0;
  for (int s = 1; s <= m.steps; ++s) {
    // wait for the 3 x 3 block of tiles to have finished step s - 1: lane
    // 3 (dy + 1) + dx + 1 of warp 0 polls neighbour (dx, dy), all at once
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x, dx = lane % 3 - 1, dy = lane / 3 - 1;
      const int nx_ = bx + dx, ny_ = by + dy;
      int ok = 1;
      if (s > 1 && lane < 9 && lane != 4 && nx_ >= 0 && ny_ >= 0 && nx_ < tx && ny_ < tyn) {
        const unsigned* f = m.flags + ny_ * tx + nx_;
        const unsigned long long t0 = global_timer_ns();
        unsigned polls = 0;
        while (ld_acquire(f) < (unsigned)(s - 1)) {
          if (ld_acquire(m.abort)) {
            ok = 0;
            break;
          }
          if (global_timer_ns() - t0 > 1000000000ull || ++polls > (1u << 24)) {
            atomicOr(a.err, FK_DEVERR_TIMEOUT);
            atomicExch(m.abort, 1u);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
      }
      ok = __all_sync(0xffffffffu, ok);
      if (lane == 0) go = ok;
    }
    __syncthreads();  // (orders every thread's staging after the acquires)
    if (!go) break;
    const int n = m.n_from - s;
    const bool odd = (m.steps - s) & 1;  // (selects, not an indexed parameter array)
    const float* src = s == 1 ? m.u_first : (odd ? m.buf[0] : m.buf[1]);
    float* dst = odd ? m.buf[1] : m.buf[0];
    const float2 e = m.e12[n];  // (e1, e2) at t_n
    masked_tile<Q, W, false, PAIR>(a, src, dst, e.x, e.y, bx, by, smem, bad);
    __syncthreads();  // every store of the tile is issued
    // the release is cumulative: it publishes the stores the barrier ordered before it
    if (threadIdx.x == 0 && by * tx + bx != m.silent) st_release(m.flags + by * tx + bx, (unsigned)s);
  }
  if (bad) atomicOr(a.err, FK_DEVERR_RANGE);
}

// Variant 3 (two nodes per thread, 2 CTAs/SM) is built for W = 7 only, the
// one width where a GB300 measured it ahead of one node per thread (the
// 1025 x 513 march: 40.2 against 40.5 ms for the best other variant).  At
// W = 5 the extra row's multiply-adds outweigh the shared reads saved
// (the kernel is issue-bound: 33.5 against 32.4 ms), and at W = 9 the two
// nodes' weights no longer fit 128 registers.  The plan offers it for
// nothing else.
template <int W>
constexpr bool kPairs = W == 7;

// Several fields run the 3-CTA/SM register budget, or the paired form of
// variant 3.
template <int Q, int W, int MINB, bool PAIR>
cudaError_t launch_m(const Step2D<float>& a, cudaStream_t s) {
  const size_t smem = fk_step2dm_smem(a.ly, a.lx);
  const int nf = a.ncols > 1 ? a.ncols : 1;
  dim3 grid((a.nx - 2 + 31) / 32, (a.ny - 2 + a.ty - 1) / a.ty, nf);
  if (nf > 1) {
    if constexpr (PAIR)
      k_step2dm<Q, W, 2, true, true><<<grid, FK_THREADS, smem, s>>>(a);
    else
      k_step2dm<Q, W, 3, true><<<grid, FK_THREADS, smem, s>>>(a);
  } else {
    k_step2dm<Q, W, MINB, false, PAIR><<<grid, FK_THREADS, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// The persistent march of a single-field plan (variant 0: 3 CTAs/SM, 1: 2,
// 2: 4, 3: pairs at 2); cudaErrorCooperativeLaunchTooLarge when the tiles
// cannot all be resident at once.
template <int Q, int W>
cudaError_t launch_march_m(const Step2D<float>& a, const MaskedMarch& m, cudaStream_t s) {
  const size_t smem = fk_step2dm_smem(a.ly, a.lx);
  const dim3 grid((a.nx - 2 + 31) / 32, (a.ny - 2 + a.ty - 1) / a.ty);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(FK_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.variant == 1) return cudaLaunchKernelEx(&cfg, k_march2dm<Q, W, 2>, a, m);
  if (a.variant == 2) return cudaLaunchKernelEx(&cfg, k_march2dm<Q, W, 4>, a, m);
  if constexpr (kPairs<W>)
    if (a.variant == 3) return cudaLaunchKernelEx(&cfg, k_march2dm<Q, W, 2, true>, a, m);
  if (a.variant == 3) return cudaErrorInvalidValue;
  return cudaLaunchKernelEx(&cfg, k_march2dm<Q, W, 3>, a, m);
}

// The single-field step of register-budget variant a.variant (0: 3 CTAs/SM,
// 1: 2, 2: 4, 3: pairs at 2).
template <int Q, int W>
cudaError_t launch_v(const Step2D<float>& a, cudaStream_t s) {
  switch (a.variant) {
    case 1: return launch_m<Q, W, 2, false>(a, s);
    case 2: return launch_m<Q, W, 4, false>(a, s);
    case 3:
      if constexpr (kPairs<W>) return launch_m<Q, W, 2, true>(a, s);
      else return cudaErrorInvalidValue;
    default: return launch_m<Q, W, 3, false>(a, s);
  }
}

// Whether every tile of the persistent march can be resident at once.
template <int Q, int W>
bool march_fits_m(const Step2D<float>& a) {
  const size_t smem = fk_step2dm_smem(a.ly, a.lx);
  const int tiles = ((a.nx - 2 + 31) / 32) * ((a.ny - 2 + a.ty - 1) / a.ty);
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  cudaError_t e = cudaErrorInvalidValue;
  if (a.variant == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march2dm<Q, W, 2>, FK_THREADS, smem);
  else if (a.variant == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march2dm<Q, W, 4>, FK_THREADS, smem);
  else if (a.variant == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march2dm<Q, W, 3>, FK_THREADS, smem);
  if constexpr (kPairs<W>)
    if (a.variant == 3)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march2dm<Q, W, 2, true>,
                                                        FK_THREADS, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (int64_t)per * sms >= tiles;
}

template <typename F>
cudaError_t big_smem(F* f, int bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int Q, int W>
cudaError_t attr_m() {
  const int big = 227 * 1024;
  // (the persistent march keeps a word of static shared memory beside the dynamic part)
  const int bigm = big - 1024;
  cudaError_t e = big_smem(k_step2dm<Q, W, 3, false>, big);
  if (e == cudaSuccess) e = big_smem(k_step2dm<Q, W, 2, false>, big);
  if (e == cudaSuccess) e = big_smem(k_step2dm<Q, W, 4, false>, big);
  if (e == cudaSuccess) e = big_smem(k_step2dm<Q, W, 3, true>, big);
  if (e == cudaSuccess) e = big_smem(k_march2dm<Q, W, 3>, bigm);
  if (e == cudaSuccess) e = big_smem(k_march2dm<Q, W, 2>, bigm);
  if (e == cudaSuccess) e = big_smem(k_march2dm<Q, W, 4>, bigm);
  if constexpr (kPairs<W>) {
    if (e == cudaSuccess) e = big_smem(k_step2dm<Q, W, 2, false, true>, big);
    if (e == cudaSuccess) e = big_smem(k_step2dm<Q, W, 2, true, true>, big);
    if (e == cudaSuccess) e = big_smem(k_march2dm<Q, W, 2, true>, bigm);
  }
  return e;
}

}  // namespace

// The entry points of one (rule size, window width): the single-field step,
// the persistent march, its residency test and the shared-memory opt-in.
#define FK_DEFINE_MASKED_QW(QQ, WW)                                                         \
  cudaError_t fk_launch_step2dm_q##QQ##w##WW(const Step2D<float>& a, cudaStream_t s) {      \
    return launch_v<QQ, WW>(a, s);                                                          \
  }                                                                                         \
  cudaError_t fk_launch_march2dm_q##QQ##w##WW(const Step2D<float>& a, const MaskedMarch& m, \
                                              cudaStream_t s) {                             \
    return launch_march_m<QQ, WW>(a, m, s);                                                 \
  }                                                                                         \
  bool fk_march2dm_fits_q##QQ##w##WW(const Step2D<float>& a) {                              \
    return march_fits_m<QQ, WW>(a);                                                         \
  }                                                                                         \
  cudaError_t fk_prepare_masked_q##QQ##w##WW() { return attr_m<QQ, WW>(); }
