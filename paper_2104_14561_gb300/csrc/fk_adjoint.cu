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
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "fk_internal.h"

namespace {

template <typename T>
struct AdjArgs {
  Step2D<T> s;      // u_in = u^{n+1}; staging and drift as in the forward step
  const T* lam;     // lambda^n
  T* mu;            // 3 J accumulators (zero on entry): [u; h u_x; h u_y] parts
  double* dth;      // 4 parameter derivatives (accumulated)
  // d(shift in cells)/d theta_k = ax_k + cn_k g (x) and ay_k + cn_k g (y):
  // cellular flow: ax_A = kx cy sx1, ax_eps = kx cy st sx2, ax_om = kx cy sw sx2
  //                (and 2 st, 2 sw with cx2 for y); constant drift: ax_b1 = dt/hx
  T st, sw;         // sin(omega t_n), eps t_n cos(omega t_n)
  T cbx, cby;       // constant drift: dt / h per axis
  T cn;             // d sigma / d theta_3 divided by sigma
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

// d(scaled slope at m)/d u_i along one line, with the end rule
template <typename T>
__device__ __forceinline__ T dslope(const T* u, int64_t stride, int n, int m, int i) {
  int l1, l0, r1, r0;
  if (m == 0) {
    l1 = 1; l0 = 0; r1 = 2; r0 = 1;
  } else if (m == n - 1) {
    l1 = n - 1; l0 = n - 2; r1 = n - 2; r0 = n - 3;
  } else {
    l1 = m; l0 = m - 1; r1 = m + 1; r0 = m;
  }
  const T dl = u[l1 * stride] - u[l0 * stride];
  const T dr = u[r1 * stride] - u[r0 * stride];
  if (!(dl * dr > T(0))) return T(0);
  const T s = dl + dr;
  const T gl = T(2) * dr * dr / (s * s), gr = T(2) * dl * dl / (s * s);
  return gl * (T(i == l1) - T(i == l0)) + gr * (T(i == r1) - T(i == r0));
}

// lambda^{n+1}_i = mu_u[i] + sum_m mu_x[m] dD^x_m/du_i + sum_m mu_y[m] dD^y_m/du_i
template <typename T>
__global__ void k_adj_slopes_t(const T* __restrict__ u, const T* __restrict__ mu,
                               T* __restrict__ lam_out, int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || k >= ny) return;
  const int64_t J = (int64_t)nx * ny, j = (int64_t)k * nx + i;
  T acc = mu[j];
  const T* urow = u + (int64_t)k * nx;
  const T* mx = mu + J + (int64_t)k * nx;
  // slopes that read u_i: nodes i-1, i, i+1, and the end nodes within reach
  for (int m = i - 2; m <= i + 2; ++m) {
    if (m < 0 || m >= nx) continue;
    const bool reach = (m >= i - 1 && m <= i + 1) || m == 0 || m == nx - 1;
    if (!reach || mx[m] == T(0)) continue;
    acc += mx[m] * dslope(urow, 1, nx, m, i);
  }
  const T* ucol = u + i;
  const T* my = mu + 2 * J + i;
  for (int m = k - 2; m <= k + 2; ++m) {
    if (m < 0 || m >= ny) continue;
    const bool reach = (m >= k - 1 && m <= k + 1) || m == 0 || m == ny - 1;
    if (!reach || my[(int64_t)m * nx] == T(0)) continue;
    acc += my[(int64_t)m * nx] * dslope(ucol, nx, ny, m, k);
  }
  lam_out[j] = acc;
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

template <typename T>
fk_status adj_step(fk_plan* p, int n, const void* u_in, const void* lam, void* lam_out,
                   double* dth, int ty, cudaStream_t s) {
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
  g.lam = (const T*)lam;
  g.mu = (T*)p->adj_mu;
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
  cudaError_t e = launch_adj<T>(g, p->q, s);
  if (e != cudaSuccess) return FK_ERR_CUDA;
  const dim3 b(32, 8), gr((p->grid.n[0] + 31) / 32, (p->grid.n[1] + 7) / 8);
  k_adj_slopes_t<T><<<gr, b, 0, s>>>((const T*)u_in, (const T*)p->adj_mu, (T*)lam_out,
                                     p->grid.n[0], p->grid.n[1]);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemsetAsync(p->adj_mu, 0, (size_t)3 * p->J * sizeof(T), s);
  return e == cudaSuccess ? FK_OK : FK_ERR_CUDA;
}

}  // namespace

extern "C" fk_status fk_adjoint(fk_plan* p, const void* u_terminal, const double* cotangent_u0,
                                double* dtheta, void* du_terminal, int K, cudaStream_t s) {
  if (!p || !cotangent_u0 || K < 1) return FK_ERR_INVALID_ARG;
  if (p->grid.dim != 2 || p->path != FK_PATH_MATRIX_FREE) return FK_ERR_UNSUPPORTED;
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
  // workspace: checkpoints (M+1), a segment (K), lambda x2, mu (3 fields), dtheta
  const int64_t need = (int64_t)(M + 1 + K + 2 + 3) * fb + 64;
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
  char* seg = base + (int64_t)(M + 1) * fb;
  void* lam[2] = {seg + (int64_t)K * fb, seg + (int64_t)(K + 1) * fb};
  p->adj_mu = seg + (int64_t)(K + 2) * fb;
  double* dth = dtheta ? dtheta : (double*)(seg + (int64_t)(K + 5) * fb);
  auto slot = [&](int n) { return n == N ? M : n / K; };  // n == N or n % K == 0

  // forward pass with checkpoints
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
  if (cudaMemsetAsync(p->adj_mu, 0, (size_t)3 * fb, s) != cudaSuccess ||
      cudaMemsetAsync(dth, 0, 4 * sizeof(double), s) != cudaSuccess)
    return FK_ERR_CUDA;
  // lambda^0 = g
  int cur = 0;
  {
    const int blocks = (int)((p->J + 255) / 256 < 152 * 16 ? (p->J + 255) / 256 : 152 * 16);
    if (p->prec == FK_FP32)
      k_cast_in<float><<<blocks, 256, 0, s>>>(cotangent_u0, (float*)lam[cur], p->J);
    else
      k_cast_in<double><<<blocks, 256, 0, s>>>(cotangent_u0, (double*)lam[cur], p->J);
    if (cudaGetLastError() != cudaSuccess) return FK_ERR_CUDA;
  }
  // backward over segments [mK, top)
  for (int m = 0; m < M; ++m) {
    const int lo = m * K, top = (m + 1) * K < N ? (m + 1) * K : N;
    // recompute u^{top-1} .. u^{lo+1} into the segment buffer
    const void* s2 = ckpt(slot(top));
    for (int n = top - 1; n >= lo + 1; --n) {
      void* dst = seg + (int64_t)(n - lo - 1) * fb;
      fk_status st = fk_enqueue_step(p, n, s2, dst, nullptr, s);
      if (st != FK_OK) return st;
      s2 = dst;
    }
    for (int n = lo; n < top; ++n) {
      const void* u_in = (n + 1 == top) ? ckpt(slot(top)) : (const void*)(seg + (int64_t)(n - lo) * fb);
      fk_status st = p->prec == FK_FP32
                         ? adj_step<float>(p, n, u_in, lam[cur], lam[cur ^ 1], dth, ty, s)
                         : adj_step<double>(p, n, u_in, lam[cur], lam[cur ^ 1], dth, ty, s);
      if (st != FK_OK) return st;
      cur ^= 1;
    }
  }
  if (du_terminal && fk_launch_copy(du_terminal, lam[cur], fb, s) != cudaSuccess) return FK_ERR_CUDA;
  return FK_OK;
}
