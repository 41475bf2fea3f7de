// Internal declarations shared by the translation units of libfk_gb300.
// Nothing here is part of the C ABI (include/fk.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fk.h"

#define FK_MAXQ 16      // largest 1D rule a plan accepts (dim = 1)
#define FK_MAXQ_2D 8    // largest rule per axis for dim = 2
#define FK_THREADS 256  // threads per CTA of the march kernels

// Device error word bits (fk_last_device_error).
#define FK_DEVERR_RANGE 1u    // a shifted point fell outside its tile halo
#define FK_DEVERR_TIMEOUT 2u  // a bounded grid-barrier wait gave up

// Named NVTX range over a host scope (profiler timelines; free when no
// profiler is attached: NVTX v3 is header-only and loads a tool on demand).
#include <nvtx3/nvToolsExt.h>
struct FkRange {
  explicit FkRange(const char* name) { nvtxRangePushA(name); }
  ~FkRange() { nvtxRangePop(); }
  FkRange(const FkRange&) = delete;
  FkRange& operator=(const FkRange&) = delete;
};

// Two- and four-component records aligned for single vector shared-memory
// accesses (16 B for float4-like, 32 B for double4-like).
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
  T x, y;
};

// Everything one 2D step kernel needs, passed by value.  All lengths are in
// cells of the uniform mesh ("index space"): node i sits at lo + i h, and a
// shifted point is i + delta with delta = b dt / h + sigma sqrt(2 dt) a / h.
template <typename T>
struct Step2D {
  const T* u_in;   // u^{n+1}
  T* u_out;        // u^n
  T* snap;         // optional second copy of u^n (snapshot), or nullptr
  int nx, ny;
  int tx, ty;      // output tile (interior nodes) per CTA: tx = 32, ty = 8 m
  int variant;     // register-budget variant (FP32 direct and row window: 0 -> 4
                   // CTAs/SM, 1 -> 3; masked window: 0 -> 3, 1 -> 2, 2 -> 4,
                   // 3 -> 2 with two nodes of a column per thread)
  int hx, hy;      // halo in cells
  int lx, ly;      // staged value tile: tx + 2 hx + 2, ty + 2 hy + 2
  int lyr;         // odd pitch of the record tiles: column pitch of the column-major
                   // tiles (modes 0, 1), row pitch of the row-major tile (mode 2)
  int family;
  // drift in cells: cellular flow  dx = kx cos(pi y)(A sin(pi x) + e1 sin(2 pi x))
  //                                dy = ky sin(pi y)(A cos(pi x) + e2 cos(2 pi x))
  //                 constant drift dx = cdx, dy = cdy
  T kx, ky, A, e1, e2, cdx, cdy;
  const T* col_tab;  // per column i: sin(pi x), sin(2 pi x), cos(pi x), cos(2 pi x)
  const T* row_tab;  // per row k: cos(pi y), sin(pi y)
  T gx[FK_MAXQ_2D], gy[FK_MAXQ_2D], w[FK_MAXQ_2D];  // sigma sqrt(2dt) a_q / h, w_q
  unsigned* err;
  // row split between the direct and the window kernel (win > 0): the
  // window kernel takes rows [row_lo, row_hi), the direct kernel (mode 1)
  // the bands [1, row_lo) and [row_hi, ny-1), nb_lo tiles for the lower one
  // (mode 2: the masked tensor-window kernel on every interior row; win is
  // then its window width W on both axes and hx, hy its halo)
  int mode, win, row_lo, row_hi, nb_lo;
  int wm[FK_MAXQ_2D];  // floor(gy_q - gy_0): y-cell offset of point q in the window
  T wmf[FK_MAXQ_2D];   // the same offsets as T (mode 2: equal on both axes)
  // Several independent fields marched by one launch (the horizons of
  // Algorithm 1, Sec. 3.2): blockIdx.z selects the field at offset
  // z * zstride of u_in and u_out, ncols fields (1 and zstride 0 for one
  // field; snapshots are not taken then).
  int64_t zstride;
  int ncols;
  __device__ __forceinline__ const T* in() const { return u_in + (int64_t)blockIdx.z * zstride; }
  __device__ __forceinline__ T* out() const { return u_out + (int64_t)blockIdx.z * zstride; }
  // Periodic x (Sec. 4.2's example): node nx-1 is node 0, the period is
  // nx - 1 nodes, staging and slopes wrap, no point exits through x, and
  // only the y faces are boundary nodes (direct kernel only).
  int px;
  // Non-uniform axes (direct kernel only): node coordinates xc[nx], yc[ny];
  // drift and point offsets (kx, ky, cdx, cdy, gx, gy) are then physical
  // lengths, not cells, and [blo, bhi] is the box.
  int nu;
  const T* xc;
  const T* yc;
  T blo[2], bhi[2];
  // masked tensor window (mode 2): index of the cell-offset pattern m_q
  // among those of (Q, W) (fk_mpat), and g_q - m_q per axis
  int mpat;
  T gmx[FK_MAXQ_2D], gmy[FK_MAXQ_2D];
};

// Cell-offset patterns of the masked tensor-window kernel.  With the 1D
// Gauss-Hermite abscissae a_q of the rule of Q points and c = sigma
// sqrt(2 dt) / h (the spread of the points in cells), point q lies
// m_q = floor(c (a_q - a_0)) cells after point 0's cell, up to one more
// cell; the window spans W = m_{Q-1} + 3 nodes.  The rows below list every
// pattern m that some c > 0 produces with W <= 9, for Q = 4, 6 and 8
// (found by walking c across the breakpoints j / (a_q - a_0)), numbered
// k = 0, 1, ... within each (Q, W).  fk_mpat returns m_q of pattern k of
// (Q, W), or -1 past the last pattern; fk_npat the number of patterns.
__host__ __device__ constexpr int fk_mpat(int Q, int W, int k, int q) {
  const signed char t[57][11] = {
      {4, 3, 0, 0, 0, 0, 0},          {4, 4, 0, 0, 0, 0, 1},          {4, 4, 1, 0, 0, 1, 1},
      {4, 5, 0, 0, 0, 1, 2},          {4, 5, 1, 0, 1, 1, 2},          {4, 6, 0, 0, 1, 1, 3},
      {4, 6, 1, 0, 1, 2, 3},          {4, 7, 0, 0, 1, 2, 4},          {4, 7, 1, 0, 1, 3, 4},
      {4, 8, 0, 0, 1, 3, 5},          {4, 8, 1, 0, 2, 3, 5},          {4, 9, 0, 0, 2, 3, 6},
      {4, 9, 1, 0, 2, 4, 6},
      {6, 3, 0, 0, 0, 0, 0, 0, 0},    {6, 4, 0, 0, 0, 0, 0, 0, 1},    {6, 4, 1, 0, 0, 0, 0, 1, 1},
      {6, 4, 2, 0, 0, 0, 1, 1, 1},    {6, 5, 0, 0, 0, 0, 1, 1, 2},    {6, 5, 1, 0, 0, 1, 1, 1, 2},
      {6, 5, 2, 0, 0, 1, 1, 2, 2},    {6, 6, 0, 0, 0, 1, 1, 2, 3},    {6, 6, 1, 0, 0, 1, 2, 2, 3},
      {6, 6, 2, 0, 0, 1, 2, 3, 3},    {6, 7, 0, 0, 0, 1, 2, 3, 4},    {6, 7, 1, 0, 1, 1, 2, 3, 4},
      {6, 7, 2, 0, 1, 2, 2, 3, 4},    {6, 8, 0, 0, 1, 2, 2, 3, 5},    {6, 8, 1, 0, 1, 2, 3, 3, 5},
      {6, 8, 2, 0, 1, 2, 3, 4, 5},    {6, 9, 0, 0, 1, 2, 3, 4, 6},    {6, 9, 1, 0, 1, 2, 3, 5, 6},
      {6, 9, 2, 0, 1, 2, 4, 5, 6},
      {8, 3, 0, 0, 0, 0, 0, 0, 0, 0, 0}, {8, 4, 0, 0, 0, 0, 0, 0, 0, 0, 1},
      {8, 4, 1, 0, 0, 0, 0, 0, 0, 1, 1}, {8, 4, 2, 0, 0, 0, 0, 0, 1, 1, 1},
      {8, 4, 3, 0, 0, 0, 0, 1, 1, 1, 1}, {8, 5, 0, 0, 0, 0, 0, 1, 1, 1, 2},
      {8, 5, 1, 0, 0, 0, 1, 1, 1, 1, 2}, {8, 5, 2, 0, 0, 0, 1, 1, 1, 2, 2},
      {8, 5, 3, 0, 0, 0, 1, 1, 2, 2, 2}, {8, 6, 0, 0, 0, 0, 1, 1, 2, 2, 3},
      {8, 6, 1, 0, 0, 1, 1, 1, 2, 2, 3}, {8, 6, 2, 0, 0, 1, 1, 2, 2, 2, 3},
      {8, 6, 3, 0, 0, 1, 1, 2, 2, 3, 3}, {8, 7, 0, 0, 0, 1, 1, 2, 2, 3, 4},
      {8, 7, 1, 0, 0, 1, 1, 2, 3, 3, 4}, {8, 7, 2, 0, 0, 1, 2, 2, 3, 3, 4},
      {8, 7, 3, 0, 0, 1, 2, 2, 3, 4, 4}, {8, 8, 0, 0, 0, 1, 2, 2, 3, 4, 5},
      {8, 8, 1, 0, 0, 1, 2, 3, 3, 4, 5}, {8, 8, 2, 0, 0, 1, 2, 3, 4, 4, 5},
      {8, 8, 3, 0, 0, 1, 2, 3, 4, 5, 5}, {8, 9, 0, 0, 0, 1, 2, 3, 4, 5, 6},
      {8, 9, 1, 0, 1, 1, 2, 3, 4, 5, 6}, {8, 9, 2, 0, 1, 2, 2, 3, 4, 5, 6},
      {8, 9, 3, 0, 1, 2, 3, 3, 4, 5, 6}};
  for (int r = 0; r < 57; ++r)
    if (t[r][0] == Q && t[r][1] == W && t[r][2] == k) return (q >= 0 && q < Q) ? t[r][3 + q] : -1;
  return -1;
}
__host__ __device__ constexpr int fk_npat(int Q, int W) {
  int n = 0;
  while (fk_mpat(Q, W, n, 0) >= 0) ++n;
  return n;
}

template <typename T>
struct Step1D {
  const T* u_in;
  T* u_out;
  T* snap;
  int nx;
  int tx;   // output nodes per CTA
  int hx;   // halo in cells
  int lx;   // tx + 2 hx + 2
  T cdx;    // b dt / h
  T g[FK_MAXQ], w[FK_MAXQ];
  unsigned* err;
  int64_t zstride;  // fields marched by one launch, as in Step2D
  int ncols;
  int nu;           // non-uniform mesh (per-step kernel only): coordinates xc,
  const T* xc;      // physical cdx and g, the box [blo, bhi]
  T blo, bhi;
  __device__ __forceinline__ const T* in() const { return u_in + (int64_t)blockIdx.z * zstride; }
  __device__ __forceinline__ T* out() const { return u_out + (int64_t)blockIdx.z * zstride; }
};

// One 3D step (fk_march3d.cuh): uniform mesh, lengths in cells as in Step2D.
template <typename T>
struct Step3D {
  const T* u_in;
  T* u_out;
  T* snap;
  V4<T>* rec;        // J records {u, hx u_x, hy u_y, hz u_z} (plan workspace)
  int nx, ny, nz;
  int q;             // Gauss-Hermite points per axis
  int w3;            // window width W (3..8) on every axis
  T cd[3];           // b dt / h per axis (constant drift)
  T gs[3];           // sigma sqrt(2 dt) / h per axis
  T ga[FK_MAXQ_2D], gw[FK_MAXQ_2D];  // abscissae (ascending) and weights
  unsigned* err;
  // the runaway-electron family (FK_RUNAWAY_3D): per-node coefficients from
  // the node coordinates x_m = lo[m] + i h[m] (FP64, as the mesh is defined)
  int family;
  double lo[3], h[3];
  double rp[11];     // E, tau, Z, delta, nu_ee, v_T, r_D, W, Delta_p, V_0, D_0
  T dt, sq2dt;       // dt and sqrt(2 dt)
  // face rules per axis (lower, upper): 0 exit value 0, 1 exit value 1,
  // 2 reflect; and the nodes the scheme updates: first[m] .. first[m] +
  // count[m] - 1 (the nodes of reflecting faces included)
  int face[3][2];
  int first[3], count[3];
  // non-uniform axes (nu): node coordinates per axis in T (positions of the
  // shifted points, cells, widths) and in FP64 (the runaway coefficients);
  // cd and gs are then physical lengths b dt and sigma sqrt(2 dt), the
  // records hold raw derivatives {u, u_x, u_y, u_z}
  int nu;
  const T* xc[3];
  const double* xd[3];
  // the runaway model: the per-node shift and scale (sh[0..2], gs[0..2],
  // six planes of J values, plan workspace) that k_step3d reads; filled once
  // per plan by fk_launch_coef3d for the static model, and by the step itself
  // (coef_per_step) for the quench variant, whose constants change with t_n
  const T* coef;
  int coef_per_step;
};
template <typename T>
cudaError_t fk_launch_step3d(const Step3D<T>& a, cudaStream_t s);
// The per-node runaway coefficients of every node the scheme updates into
// coef (6 J values), from the same device code the step evaluates them with.
template <typename T>
cudaError_t fk_launch_coef3d(const Step3D<T>& a, T* coef, cudaStream_t s);
// The terminal indicator of a 3D plan: 1 on the faces whose exit value is
// 1, 0 elsewhere.
template <typename T>
cudaError_t fk_launch_chi3d(const Step3D<T>& a, T* u, cudaStream_t s);
#define FK_MAXW_3D 8
#define FK_FACE_EXIT0 0
#define FK_FACE_EXIT1 1
#define FK_FACE_REFLECT 2

// Shared memory bytes of one 2D step CTA (nu: plus the staged node
// coordinates of a non-uniform mesh).
size_t fk_step2d_smem(int lx, int ly, int lyr, int elem, int nu = 0);
size_t fk_step1d_smem(int lx, int elem, int nu = 0);

// Launchers (fk_march.cu).  Return cudaGetLastError().
template <typename T>
cudaError_t fk_launch_step2d(const Step2D<T>& a, int q, cudaStream_t s);
template <typename T>
cudaError_t fk_launch_step1d(const Step1D<T>& a, int q, cudaStream_t s);
// Opt the step kernels of this (dim, q, precision) into large dynamic shared
// memory; called once at plan creation, never during stream capture.
cudaError_t fk_prepare_step_kernels(int dim, int q, int elem);
// Whether a window kernel with W rows exists for rule size q (FP32 only).
bool fk_window_available(int q, int w);
// The masked tensor-window kernel (fk_window.cu, FP32): launcher, shared
// memory of one CTA, availability for (q, W), and the large-shared-memory
// opt-in (plan creation only).
cudaError_t fk_launch_step2dm(const Step2D<float>& a, int q, cudaStream_t s);
size_t fk_step2dm_smem(int ly, int lx);  // ly staged rows of lx nodes
// staged columns of a masked-window tile: 32 output columns, the halo on
// both sides, one node on each side for the slopes, and one more column
// when W is odd (the window is read in pairs of columns)
int fk_step2dm_lx(int hx, int w);
bool fk_masked_available(int q, int w);
// The FP64 masked tensor-window kernel (fk_window64.cu): launcher, shared
// memory of one CTA (ly staged rows of lx nodes) and the large-shared-memory
// opt-in (plan creation only).
cudaError_t fk_launch_step2dm64(const Step2D<double>& a, int q, cudaStream_t s);
size_t fk_step2dm64_smem(int ly, int lx);
cudaError_t fk_prepare_masked64(int q);
// index k of the pattern m[0..q-1] among those of (q, w), or -1
int fk_masked_pattern(int q, int w, const int* m);
cudaError_t fk_prepare_masked_kernels(int q);
// The persistent march of the FP32 masked kernel (fk_window.cuh): the steps
// n_from-1 .. n_from-steps of one field in one cooperative launch, one CTA
// per tile; step m reads u_first (m = 1) or buf[(steps - m + 1) & 1] and
// writes buf[(steps - m) & 1].  flags (one word per tile) and abort must be
// zero at launch.
struct MaskedMarch {
  const float* u_first;
  float* buf[2];
  const float2* e12;  // per time index n: the cellular flow's eps sin(omega t_n) factors
  unsigned* flags;
  unsigned* abort;
  int n_from, steps;
  int silent;  // tile that never publishes its step count (test hook; -1 none)
};
cudaError_t fk_launch_march2dm(const Step2D<float>& a, const MaskedMarch& m, int q,
                               cudaStream_t s);
bool fk_march2dm_fits(const Step2D<float>& a, int q);  // all tiles resident at once
// Every (rule size, window width) the FP32 masked kernels are built for, and
// their entry points (fk_window_q*.cu, a few widths per translation unit so
// that the parallel build stays short).
#define FK_MASKED_ALL(X)                                  \
  X(4, 3) X(4, 4) X(4, 5) X(4, 6) X(4, 7) X(4, 8) X(4, 9) \
  X(6, 3) X(6, 4) X(6, 5) X(6, 6) X(6, 7) X(6, 8) X(6, 9) \
  X(8, 3) X(8, 4) X(8, 5) X(8, 6) X(8, 7) X(8, 8) X(8, 9)
#define FK_DECLARE_MASKED_QW(QQ, WW)                                                        \
  cudaError_t fk_launch_step2dm_q##QQ##w##WW(const Step2D<float>& a, cudaStream_t s);       \
  cudaError_t fk_launch_march2dm_q##QQ##w##WW(const Step2D<float>& a, const MaskedMarch& m, \
                                              cudaStream_t s);                              \
  bool fk_march2dm_fits_q##QQ##w##WW(const Step2D<float>& a);                               \
  cudaError_t fk_prepare_masked_q##QQ##w##WW();
FK_MASKED_ALL(FK_DECLARE_MASKED_QW)
// (Q, W) pairs of the masked-window adjoint kernel (fk_adjoint.cu): the
// window form pays off while W^2 cells stay below the direct form's 4 Q^2
// corner reads and its weights fit in registers.
#define FK_MASKED_LIST(X)                                                  \
  X(4, 3) X(4, 4) X(4, 5) X(4, 6) X(4, 7)                                  \
  X(6, 3) X(6, 4) X(6, 5) X(6, 6) X(6, 7) X(6, 8) X(6, 9)                  \
  X(8, 3) X(8, 4) X(8, 5) X(8, 6) X(8, 7) X(8, 8) X(8, 9)

// 1D march resident in one CTA (fk_march1d.cu): all `steps` steps of
// Scheme 1 from u_in (NULL = chi) into u_out (may alias u_in), snapshots
// every `stride` steps when snaps != NULL.
size_t fk_march1d_smem(int nx, int elem);
template <typename T>
cudaError_t fk_launch_march1d(const Step1D<T>& a, int q, const T* u_in, T* u_out, T* snaps,
                              int stride, int steps, cudaStream_t s);
cudaError_t fk_prepare_march1d(int q, int elem);
// The same march over a cluster of `ctas` CTAs (distributed shared memory).
template <typename T>
cudaError_t fk_launch_march1d_cluster(const Step1D<T>& a, int q, int ctas, const T* u_in,
                                      T* u_out, T* snaps, int stride, int steps, cudaStream_t s);
int fk_prepare_march1d_cluster(int q, int elem);
// The terminal indicator chi: 1 on the boundary nodes (with px, the x faces
// are identified and only the y faces are boundary), 0 elsewhere; nz is the
// third extent of a 3D mesh.
cudaError_t fk_launch_fill_chi(void* u, int dim, int nx, int ny, int elem, cudaStream_t s,
                               int px = 0, int nz = 1);
// Starting fields of the horizon march: field c = 1..nfields (at offset
// (c - 1) J) of buffer `odd` for odd c and of buffer `even` for even c gets
// src (J values) or, with src NULL, the terminal indicator.
cudaError_t fk_launch_fill_fields(void* even, void* odd, const void* src, int dim, int nx, int ny,
                                  int elem, int nfields, cudaStream_t s, int px = 0, int nz = 1);
cudaError_t fk_launch_copy(void* dst, const void* src, int64_t bytes, cudaStream_t s);

struct fk_plan {
  fk_grid grid;
  fk_region region;
  fk_coeffs coeffs;
  int q;
  double dt;
  int n_steps;
  fk_precision prec;
  fk_path path;
  int device;
  int elem;          // 4 or 8
  int64_t J, J_int;
  double h[3];
  double reach[3];
  int halo[3], tile[3];
  int variant;       // register-budget variant of the 2D step kernel
  int win;           // rows of the window kernel in use (0: direct kernel only)
  int win_max;       // rows the window kernel needs (0: not eligible)
  int win_row_lo, win_row_hi;
  int wm[FK_MAXQ_2D];
  int mwin;          // window width of the masked tensor-window kernel (0: not eligible)
  int mwm[FK_MAXQ_2D];  // its cell offsets floor(g_q - g_0), equal on both axes
  int mhalo[2];      // its halo per axis
  int mpat;          // index of its cell-offset pattern among those of (q, mwin)
  // the persistent march of the masked kernel (fk_window.cuh): whether
  // whole marches use it (1), its tile flags and abort word, and the
  // per-step drift factors; batch: the batched call forbids it while its
  // plans run concurrently
  int persist;
  unsigned* mflags;
  int64_t mflags_n;
  float2* me12;
  int no_persist;
  int g_persist;     // the cached graph was built with the persistent march
  int use_masked;    // the masked kernel is the step kernel
  int resident1d;    // 1D: 0 one launch per step, 1 the whole march in one CTA,
                     // 2 in one cluster of cluster1d CTAs (fk_march1d.cu)
  int cluster1d;
  double gh_a[FK_MAXQ], gh_w[FK_MAXQ];
  // device memory owned by the plan
  void* scratch;     // one field
  void* col_tab;     // 4 * nx values of the plan precision
  void* row_tab;     // 2 * ny values
  unsigned* d_err;
  int64_t workspace_bytes;
  cudaStream_t cap_stream;  // private stream used for graph capture
  // CUDA graph cache for fk_solve
  cudaGraphExec_t graph;
  const void* g_in;
  void* g_out;
  void* g_snap;
  int g_stride;
  // CSR path (fk_csr.cu)
  int64_t csr_nnz;       // stored entries of A = Q Psi: three per record
  int64_t* csr_rowptr;  // J + 1 row offsets, in records
  void* csr_val;     // csr_nnz / 3 records {node, weights of u, h u_x, h u_y}
  void* csr_c;       // J: exit weight constant per row
  void* stack;       // 4 J: {u, h u_x, h u_y, 0} per node for the CSR product
  // batched persistent march (fk_batched.cu)
  void* batch_rec;   // 6 J values: slope records of this instance
  void* batch_work;  // BatchWork of a batch whose first plan is this one
  int batch_grid;    // CTAs of the last batched launch
  int periodic_x;    // the x faces are identified (region FK_PERIODIC_X)
  int nu;            // non-uniform axes: node coordinates per axis
  double* hcoord[3]; // host copies (malloc) and device copies in the plan's precision
  void* dcoord[3];
  void* dcoord64[3]; // d = 3, FP32 plans: FP64 device copies (runaway coefficients)
  // d = 3: the node records of the step and the window width
  void* rec3d;
  void* coef3d;      // the static runaway model's per-node coefficients (6 J values)
  int w3;
  // fk_solve_host: the device copy of the host field (one field, on first use)
  void* host_io;
  // fk_solve_horizons: the second buffer of the N horizon fields
  void* hz_ws;
  int64_t hz_bytes;
  // adjoint (fk_adjoint.cu): checkpoints, segment, lambda, mu, dtheta
  void* adj_ws;
  int64_t adj_bytes;
  void* adj_mu;      // two buffers of 3 J accumulators inside adj_ws
  int adj_ty;        // tile height of the masked-window adjoint (0: per-point scatter)
  int adj_kernel;    // backward form of the last fk_adjoint: 0 none, 1 scatter, 2 masked
  void* adj_tab;     // piecewise-cubic weight tables of the masked adjoint (device, float4)
  float adj_break[2][FK_MAXQ_2D];  // their piece boundaries per axis, unused ones 2
  float adj_last[2];               // g_{Q-1} - g_0 per axis
  // fk_adjoint_kernel_times: CUDA events around each backward-step kernel
  // launch of the recorded fk_adjoint calls (pairs; host array)
  int adj_rec;        // recording on
  cudaEvent_t* adj_ev;
  int adj_ev_cap;     // events created
  int adj_ev_used;    // events recorded by the last fk_adjoint
  // the segment recompute runs on its own stream (created on first use),
  // ordered by events: forward pass done, segment recomputed (per buffer),
  // segment's backward steps done (per buffer)
  cudaStream_t adj_s2;
  cudaEvent_t adj_sev[5];
  int adj_sev_n;      // events of adj_sev created
};

void fk_batch_release(fk_plan* p);
// Strategy of the last fk_solve_batched that plan p led (0 none, 1 the
// persistent kernel, 2 concurrent single-plan graphs).
int fk_batch_mode(const fk_plan* p);

// Step launchers that fill the argument struct from the plan (fk_plan.cu).
fk_status fk_enqueue_step(fk_plan* p, int n, const void* u_in, void* u_out, void* snap,
                          cudaStream_t s);
// The same step for nfields fields at J-value spacing (u_in and u_out point
// at the first), one launch (matrix-free path only).
fk_status fk_enqueue_step_fields(fk_plan* p, int n, const void* u_in, void* u_out, int nfields,
                                 cudaStream_t s);
void fk_fill_step2d_f32(const fk_plan* p, int n, Step2D<float>* a);
void fk_fill_step2d_f64(const fk_plan* p, int n, Step2D<double>* a);

// Device allocation through the plan's accounting.  Fault injection for
// tests: with FK_TEST_FAIL_ALLOC=n set, the n-th allocation after the value
// was set fails with FK_ERR_OOM (the count restarts when the value changes).
fk_status fk_dev_alloc(fk_plan* p, void** ptr, size_t bytes);
void fk_dev_free(void* ptr);

// CSR path (fk_csr.cu).
fk_status fk_csr_assemble(fk_plan* p, cudaStream_t s);
fk_status fk_csr_step(fk_plan* p, const void* u_in, void* u_out, void* snap, cudaStream_t s);
