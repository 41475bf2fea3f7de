// Assembled-CSR path for coefficients that do not depend on t.
//
// The step of Scheme 1 is u^n = Q Psi^n F^n u^{n+1} (Eq. (e36)): F^n maps
// u to the stacked vector X = [u; h u_x; h u_y] (the PCHIP slopes of
// Eq. (e300), scaled by the mesh width), Psi^n interpolates X at the shifted
// points (Eq. (e34)) and Q applies the quadrature weights (Eq. (e35)).  When
// b and sigma do not depend on t the product A = Q Psi is the same in every
// step, so it is assembled once and each step is a slope pass plus one
// sparse matrix-vector product, the HBM-bound form of the march.
//
// Row j of A (an interior node) factorises: with the tensor Gauss-Hermite
// points x_p (p over one axis) and y_q, and the cardinal Hermite value and
// slope functions phi_a, psi_a of node a along an axis,
//   A[j, u_ab]  = Phi_a Phi_b,  A[j, hu_x,ab] = Psi_a Phi_b,  A[j, hu_y,ab] = Phi_a Psi_b,
//   Phi_a = sum_{p inside} w_p phi_a(x_p),  Psi_a = sum_{p inside} w_p psi_a(x_p),
// over the nodes a (b) touched by the non-exiting points of that axis; the
// exit weight c_j = 1 - (sum_{p inside} w_p)(sum_{q inside} w_q) multiplies
// the exit value 1 (Eq. (e24)).  Boundary rows are empty with c_j = 1.
//
// The product is evaluated in increment form, u_j + sum A (X - u_j [u part])
// + c_j (1 - u_j), which equals A X + c exactly (the u-part of each row sums
// to 1 - c_j) but keeps FP32 rounding proportional to the per-step change.
//
// Storage: the three entries of a row that share a node ab (its u, h u_x and
// h u_y columns) are one record {column ab, A[j, u_ab], A[j, hu_x,ab],
// A[j, hu_y,ab]}: 16 B in FP32 (32 B in FP64) per three stored entries,
// instead of a 4 B column index beside every value, and one aligned vector
// load.  X is stored interleaved per node, {u, h u_x, h u_y, 0}, so that a
// record needs one gather.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cub/cub.cuh>

#include "fk_internal.h"

namespace {

const double kPi = 3.14159265358979323846264338327950288;

struct CsrAsm {
  int nx, ny, q, family;
  int64_t J;
  double kx, ky, A, cdx, cdy;  // drift in cells (as in the step kernel)
  double lox, hx, loy, hy;
  double g[2][FK_MAXQ_2D], w[FK_MAXQ_2D];
};

struct AxisW {
  int n;
  int node[2 * FK_MAXQ_2D];
  double phi[2 * FK_MAXQ_2D], psi[2 * FK_MAXQ_2D];
  double inside;  // sum of the weights of the non-exiting points
};

__device__ void axis_add(AxisW* o, int node, double ph, double ps) {
  for (int m = o->n - 1; m >= 0 && m >= o->n - 2; --m) {
    if (o->node[m] == node) {
      o->phi[m] += ph;
      o->psi[m] += ps;
      return;
    }
  }
  o->node[o->n] = node;
  o->phi[o->n] = ph;
  o->psi[o->n] = ps;
  ++o->n;
}

// Weights of one axis for a node at index k whose drift shift is d0 cells.
// Points are sorted, so touched nodes arrive in non-decreasing order.
__device__ void axis_weights(const CsrAsm& a, int axis, int k, int n, double d0, AxisW* o) {
  o->n = 0;
  o->inside = 0.0;
  for (int q = 0; q < a.q; ++q) {
    const double d = d0 + a.g[axis][q];
    if (d < -k || d > n - 1 - k) continue;  // exit along this axis
    const double fl = floor(d);
    int c = k + (int)fl;
    double t = d - fl;
    if (c > n - 2) {
      c = n - 2;
      t = 1.0;
    }
    const double w = a.w[q];
    const double h01 = t * t * (3.0 - 2.0 * t), h00 = 1.0 - h01;
    const double h10 = t * (1.0 - t) * (1.0 - t), h11 = -t * t * (1.0 - t);
    axis_add(o, c, w * h00, w * h10);
    axis_add(o, c + 1, w * h01, w * h11);
    o->inside += w;
  }
}

__device__ void row_drift(const CsrAsm& a, int i, int k, double* dx, double* dy) {
  if (a.family == FK_CELLULAR_FLOW) {
    const double x = a.lox + i * a.hx, y = a.loy + k * a.hy;
    *dx = a.kx * cos(kPi * y) * (a.A * sin(kPi * x));
    *dy = a.ky * sin(kPi * y) * (a.A * cos(kPi * x));
  } else {
    *dx = a.cdx;
    *dy = a.cdy;
  }
}

__global__ void k_csr_count(const CsrAsm a, int64_t* counts) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j > a.J) return;
  if (j == a.J) {
    counts[j] = 0;
    return;
  }
  const int i = (int)(j % a.nx), k = (int)(j / a.nx);
  if (i == 0 || k == 0 || i == a.nx - 1 || k == a.ny - 1) {
    counts[j] = 0;
    return;
  }
  double dx, dy;
  row_drift(a, i, k, &dx, &dy);
  AxisW ax, ay;
  axis_weights(a, 0, i, a.nx, dx, &ax);
  axis_weights(a, 1, k, a.ny, dy, &ay);
  counts[j] = (int64_t)ax.n * ay.n;  // records (three stored entries each)
}

// One record of a row: the column (a node index) and the weights of the
// node's u, h u_x and h u_y.  FP32: 16 B; FP64: 32 B (the column in the
// first 8 B).
template <typename T>
struct CsrRec;
template <>
struct alignas(16) CsrRec<float> {
  int col;
  float vu, vx, vy;
};
template <>
struct alignas(16) CsrRec<double> {
  int col, pad;
  double vu, vx, vy;
};

template <typename T>
__global__ void k_csr_fill(const CsrAsm a, const int64_t* rowptr, CsrRec<T>* rec, T* cvec,
                           unsigned* err) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= a.J) return;
  const int i = (int)(j % a.nx), k = (int)(j / a.nx);
  if (i == 0 || k == 0 || i == a.nx - 1 || k == a.ny - 1) {
    cvec[j] = T(1);
    return;
  }
  double dx, dy;
  row_drift(a, i, k, &dx, &dy);
  AxisW ax, ay;
  axis_weights(a, 0, i, a.nx, dx, &ax);
  axis_weights(a, 1, k, a.ny, dy, &ay);
  cvec[j] = (T)(1.0 - ax.inside * ay.inside);
  int64_t o = rowptr[j];
  const int64_t end = rowptr[j + 1];
  for (int mb = 0; mb < ay.n; ++mb) {
    for (int ma = 0; ma < ax.n; ++ma) {
      if (o >= end) {  // the count pass disagreed: never write past the row
        atomicOr(err, FK_DEVERR_RANGE);
        return;
      }
      CsrRec<T> r;
      memset(&r, 0, sizeof(r));
      r.col = (int)((int64_t)ay.node[mb] * a.nx + ax.node[ma]);
      r.vu = (T)(ax.phi[ma] * ay.phi[mb]);
      r.vx = (T)(ax.psi[ma] * ay.phi[mb]);
      r.vy = (T)(ax.phi[ma] * ay.psi[mb]);
      rec[o] = r;
      ++o;
    }
  }
}

template <typename T>
__device__ __forceinline__ T pchip_exact(T dl, T dr) {
  const T p = dl * dr;
  return p > T(0) ? (T(2) * p) / (dl + dr) : T(0);
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_16a;
};

// F^n: X = [u; h u_x; h u_y] with the PCHIP rule of Eq. (e300) and its end
// rule (node 0: (delta_0, delta_1); node n-1: (delta_{n-2}, delta_{n-3})),
// interleaved per node as {u, h u_x, h u_y, 0}.
template <typename T>
__global__ void k_csr_slopes(const T* __restrict__ u, typename Vec4<T>::type* __restrict__ X,
                             int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || k >= ny) return;
  const int64_t j = (int64_t)k * nx + i;
  const T* r = u + (int64_t)k * nx;
  T sx, sy;
  if (i == 0)
    sx = pchip_exact(r[1] - r[0], r[2] - r[1]);
  else if (i == nx - 1)
    sx = pchip_exact(r[nx - 1] - r[nx - 2], r[nx - 2] - r[nx - 3]);
  else
    sx = pchip_exact(r[i] - r[i - 1], r[i + 1] - r[i]);
  const T* c = u + i;
  const int64_t s = nx;
  if (k == 0)
    sy = pchip_exact(c[s] - c[0], c[2 * s] - c[s]);
  else if (k == ny - 1)
    sy = pchip_exact(c[(ny - 1) * s] - c[(ny - 2) * s], c[(ny - 2) * s] - c[(ny - 3) * s]);
  else
    sy = pchip_exact(c[k * s] - c[(k - 1) * s], c[(k + 1) * s] - c[k * s]);
  typename Vec4<T>::type x;
  x.x = r[i];
  x.y = sx;
  x.z = sy;
  x.w = T(0);
  X[j] = x;
}

// One warp per row; each lane takes four records per pass (128 per warp,
// about a whole row), all four record loads and then all four gathers of
// their nodes from X in flight together: a record's gather depends on its
// load, so one record per pass left each lane one L2 round trip at a time.
template <typename T>
__global__ void __launch_bounds__(256) k_csr_spmv(const int64_t* __restrict__ rowptr,
                                                  const CsrRec<T>* __restrict__ rec,
                                                  const T* __restrict__ cvec,
                                                  const typename Vec4<T>::type* __restrict__ X,
                                                  T* __restrict__ y, T* __restrict__ snap,
                                                  int64_t J) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= J) return;
  const int64_t b = rowptr[row], e = rowptr[row + 1];
  const T uj = X[row].x;
  T acc = T(0);
  for (int64_t o0 = b + lane; o0 < e; o0 += 128) {
    CsrRec<T> r[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int64_t o = o0 + 32 * m;
      if (o < e) {
        r[m] = rec[o];
      } else {  // (a zero weight on the row's own node)
        r[m].col = (int)row;
        r[m].vu = r[m].vx = r[m].vy = T(0);
      }
    }
    typename Vec4<T>::type x[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) x[m] = X[r[m].col];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc += r[m].vu * (x[m].x - uj) + r[m].vx * x[m].y + r[m].vy * x[m].z;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if (lane == 0) {
    const T c = cvec[row];
    const T un = (e == b && c == T(1)) ? T(1) : uj + acc + c * (T(1) - uj);
    y[row] = un;
    if (snap) snap[row] = un;
  }
}

}  // namespace

fk_status fk_csr_assemble(fk_plan* p, cudaStream_t s) {
  FkRange range("fk_csr_assemble");
  CsrAsm a;
  memset(&a, 0, sizeof(a));
  a.nx = p->grid.n[0];
  a.ny = p->grid.n[1];
  a.q = p->q;
  a.family = p->coeffs.family;
  a.J = p->J;
  a.kx = -kPi * p->dt / p->h[0];
  a.ky = kPi * p->dt / p->h[1];
  a.A = p->coeffs.p[0];
  a.cdx = p->coeffs.p[0] * p->dt / p->h[0];
  a.cdy = p->coeffs.p[1] * p->dt / p->h[1];
  a.lox = p->grid.lo[0];
  a.hx = p->h[0];
  a.loy = p->grid.lo[1];
  a.hy = p->h[1];
  const double sigma = p->coeffs.family == FK_CONST_DRIFT ? p->coeffs.p[3] : sqrt(2.0 * p->coeffs.p[3]);
  const double sg = sigma * sqrt(2.0 * p->dt);
  for (int q = 0; q < p->q; ++q) {
    a.g[0][q] = sg * p->gh_a[q] / p->h[0];
    a.g[1][q] = sg * p->gh_a[q] / p->h[1];
    a.w[q] = p->gh_w[q];
  }
  const int64_t J = p->J;
  fk_status st = fk_dev_alloc(p, (void**)&p->csr_rowptr, sizeof(int64_t) * (J + 1));
  if (st != FK_OK) return st;
  int64_t* counts = nullptr;
  if (cudaMalloc(&counts, sizeof(int64_t) * (J + 1)) != cudaSuccess) {
    cudaGetLastError();
    return FK_ERR_OOM;
  }
  const int tb = 256;
  const int64_t nb = (J + 1 + tb - 1) / tb;
  k_csr_count<<<(unsigned)nb, tb, 0, s>>>(a, counts);
  size_t tmp_bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, counts, p->csr_rowptr, J + 1, s);
  void* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, tmp_bytes);
  if (e == cudaSuccess)
    e = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, counts, p->csr_rowptr, J + 1, s);
  int64_t nnz = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&nnz, p->csr_rowptr + J, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  cudaFree(counts);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FK_ERR_OOM : FK_ERR_CUDA;
  }
  if (J >= ((int64_t)1 << 31)) return FK_ERR_UNSUPPORTED;  // int32 node indices
  const int64_t nrec = nnz;  // (the scan counted records)
  p->csr_nnz = 3 * nrec;     // stored entries of A: three per record
  const size_t rec_bytes = p->prec == FK_FP32 ? sizeof(CsrRec<float>) : sizeof(CsrRec<double>);
  st = fk_dev_alloc(p, &p->csr_val, rec_bytes * (size_t)(nrec > 0 ? nrec : 1));
  if (st == FK_OK) st = fk_dev_alloc(p, &p->csr_c, (size_t)p->elem * J);
  if (st == FK_OK) st = fk_dev_alloc(p, &p->stack, (size_t)p->elem * 4 * J);
  if (st != FK_OK) return st;
  if (p->prec == FK_FP32)
    k_csr_fill<float><<<(unsigned)((J + tb - 1) / tb), tb, 0, s>>>(
        a, p->csr_rowptr, (CsrRec<float>*)p->csr_val, (float*)p->csr_c, p->d_err);
  else
    k_csr_fill<double><<<(unsigned)((J + tb - 1) / tb), tb, 0, s>>>(
        a, p->csr_rowptr, (CsrRec<double>*)p->csr_val, (double*)p->csr_c, p->d_err);
  e = cudaGetLastError();
  return e == cudaSuccess ? FK_OK : FK_ERR_CUDA;
}

fk_status fk_csr_step(fk_plan* p, const void* u_in, void* u_out, void* snap, cudaStream_t s) {
  const int nx = p->grid.n[0], ny = p->grid.n[1];
  const dim3 sb(32, 8), sg((nx + 31) / 32, (ny + 7) / 8);
  const int64_t J = p->J;
  const unsigned blocks = (unsigned)((J * 32 + 255) / 256);
  if (p->prec == FK_FP32) {
    k_csr_slopes<float><<<sg, sb, 0, s>>>((const float*)u_in, (float4*)p->stack, nx, ny);
    k_csr_spmv<float><<<blocks, 256, 0, s>>>(p->csr_rowptr, (const CsrRec<float>*)p->csr_val,
                                             (const float*)p->csr_c, (const float4*)p->stack,
                                             (float*)u_out, (float*)snap, J);
  } else {
    k_csr_slopes<double><<<sg, sb, 0, s>>>((const double*)u_in, (double4_16a*)p->stack, nx, ny);
    k_csr_spmv<double><<<blocks, 256, 0, s>>>(p->csr_rowptr, (const CsrRec<double>*)p->csr_val,
                                              (const double*)p->csr_c,
                                              (const double4_16a*)p->stack, (double*)u_out,
                                              (double*)snap, J);
  }
  return cudaGetLastError() == cudaSuccess ? FK_OK : FK_ERR_CUDA;
}
