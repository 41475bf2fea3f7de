// Batched persistent march: many independent instances of Scheme 1 (uneven
// meshes and coefficients, same rule and step count) in ONE cooperative
// kernel launch that runs all N time steps.
//
// Each time step has two phases over a flat work list of 32 x 8 node tiles
// that spans every instance:
//   R: pack the PCHIP slope records of u^{n+1} (Eq. (e300)) for every node
//      into a per-instance global array, {u_c, u_{c+1}-u_c, h u'_c,
//      h u'_{c+1}} and {h u_y,c, h u_y,c+1 - h u_y,c};
//   Q: per interior node, the tensor Gauss-Hermite shifted points of
//      Eq. (e31), the exit test (Eq. (e24)), the zero-twist Hermite values
//      of Eq. (Lag11) gathered from the records (L1/L2), the quadrature sum
//      of Eq. (e304) in increment form, and the boundary value 1 (Eq. (e3)).
// A grid barrier separates the phases.  It is a bounded wait: after ~1 s
// without progress a CTA records FK_DEVERR_TIMEOUT and every CTA leaves the
// kernel at its next barrier, so a stalled launch ends instead of hanging.
//
// Records live in global memory rather than in per-tile shared memory
// because the halo of the sweep's instances ranges from 1 to ~24 cells and
// one launch has one shared-memory size; the records of the tiles an SM is
// working on stay in its L1, the rest in the 129 MB L2.
//
// A second strategy runs every instance's own CUDA-graph march (fk_solve,
// with the single-plan step kernels that stage tiles in shared memory) on a
// pool of side streams forked from and joined into the caller's stream.
// The first call for a batch shape times a few steps of both and keeps the
// faster: the persistent kernel wins when launches dominate (many small
// instances), the concurrent graphs when the per-node work does.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fk_internal.h"

namespace {

const int kTileW = 32, kTileH = 8;  // one node per thread of a 256-thread CTA
const int kMaxInst = 256;
const unsigned long long kBarrierLimitNs = 1000000000ull;  // 1 s

template <typename T>
struct BInst {
  const T* u_first;   // input of step 1 (terminal field, chi or a copy)
  T* buf[2];          // step m writes buf[(N - m) & 1]; buf[0] is the caller's output
  V4<T>* rec;         // R records, one per node
  V2<T>* srec;        // S records
  const T* col_tab;   // sin(pi x), sin(2 pi x), cos(pi x), cos(2 pi x) per column
  const T* row_tab;   // cos(pi y), sin(pi y) per row
  const T* e12;       // per step n: eps sin(omega t_n), 2 eps sin(omega t_n)
  int nx, ny, family;
  int tiles_x_all, tiles_all;  // phase R tiles (all nodes)
  int tiles_x_int, tiles_int;  // phase Q tiles (interior nodes)
  int first_r, first_q;        // offsets of this instance in the flat work lists
  T kx, ky, A, cdx, cdy;
  T gx[FK_MAXQ_2D], gy[FK_MAXQ_2D], w[FK_MAXQ_2D];
};

struct BarrierState {
  unsigned count;
  unsigned gen;
  unsigned abort;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid barrier; returns false when the launch must stop.
__device__ bool grid_barrier(BarrierState* b, unsigned expected, unsigned* err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &b->gen;
    volatile unsigned* vabort = &b->abort;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == expected - 1) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
      ok = 1;
    } else {
      const unsigned long long t0 = global_ns();
      ok = 1;
      unsigned spins = 0;
      while (*vgen == g) {
        if (*vabort) {
          ok = 0;
          break;
        }
        // two independent bounds: 1 s of global time, or 2^24 sleeps of
        // >= 64 ns should the timer not advance
        if (global_ns() - t0 > kBarrierLimitNs || ++spins > (1u << 24)) {
          atomicOr(err, FK_DEVERR_TIMEOUT);
          atomicExch(&b->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ T bpchip(T dl, T dr) {
  const T p = dl * dr;
  return p > T(0) ? (T(2) * p) / (dl + dr) : T(0);
}
template <>
__device__ __forceinline__ float bpchip<float>(float dl, float dr) {
  const float p = dl * dr;
  return p > 0.f ? __fdividef(2.f * p, dl + dr) : 0.f;
}

// Scaled slope at node g of a line with n nodes, neighbours `stride` apart.
template <typename T>
__device__ __forceinline__ T bslope(const T* __restrict__ line, int g, int n, int64_t stride) {
  const T* c = line + g * stride;
  if (g == 0) return bpchip(c[stride] - c[0], c[2 * stride] - c[stride]);
  if (g == n - 1) return bpchip(c[0] - c[-stride], c[-stride] - c[-2 * stride]);
  return bpchip(c[0] - c[-stride], c[stride] - c[0]);
}

__device__ int find_inst(const int* first, int n_inst, int item) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_batched(const BInst<T>* __restrict__ insts, int n_inst,
                                                 int n_steps, int total_r, int total_q,
                                                 unsigned expected, BarrierState* bar,
                                                 unsigned* err) {
  __shared__ int first_r[kMaxInst], first_q[kMaxInst];
  for (int m = threadIdx.x; m < n_inst; m += blockDim.x) {
    first_r[m] = insts[m].first_r;
    first_q[m] = insts[m].first_q;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
  unsigned bad = 0;
  for (int m = 1; m <= n_steps; ++m) {
    const int n = n_steps - m;
    // ---- phase R: records of u^{n+1}
    for (int item = blockIdx.x; item < total_r; item += gridDim.x) {
      const BInst<T>& I = insts[find_inst(first_r, n_inst, item)];
      const int t = item - I.first_r;
      const int i = (t % I.tiles_x_all) * kTileW + lane;
      const int k = (t / I.tiles_x_all) * kTileH + row;
      if (i > I.nx - 2 || k >= I.ny) continue;  // cells c = 0 .. nx-2
      const T* src = (m == 1) ? I.u_first : I.buf[(n_steps - m + 1) & 1];
      const int64_t j = (int64_t)k * I.nx + i;
      const T* rowp = src + (int64_t)k * I.nx;
      const T* colp0 = src + i;
      const T u0 = rowp[i], u1 = rowp[i + 1];
      V4<T> r;
      r.x = u0;
      r.y = u1 - u0;
      r.z = bslope(rowp, i, I.nx, 1);
      r.w = bslope(rowp, i + 1, I.nx, 1);
      const T dy0 = bslope(colp0, k, I.ny, I.nx);
      const T dy1 = bslope(colp0 + 1, k, I.ny, I.nx);
      V2<T> s;
      s.x = dy0;
      s.y = dy1 - dy0;
      I.rec[j] = r;
      I.srec[j] = s;
    }
    if (!grid_barrier(bar, expected, err)) return;
    // ---- phase Q: u^n at interior nodes, 1 on the boundary
    for (int item = blockIdx.x; item < total_q; item += gridDim.x) {
      const BInst<T>& I = insts[find_inst(first_q, n_inst, item)];
      const int t = item - I.first_q;
      const int i = 1 + (t % I.tiles_x_int) * kTileW + lane;
      const int k = 1 + (t / I.tiles_x_int) * kTileH + row;
      if (i > I.nx - 2 || k > I.ny - 2) continue;
      const int nx = I.nx, ny = I.ny;
      const int64_t jn = (int64_t)k * nx + i;
      const V4<T>* R = I.rec;
      const V2<T>* S = I.srec;
      const T uj = R[jn].x;
      T dx, dy;
      if (I.family == FK_CELLULAR_FLOW) {
        const T* ct = I.col_tab + 4 * (int64_t)i;
        const T* rt = I.row_tab + 2 * (int64_t)k;
        const T e1 = I.e12[2 * n], e2 = I.e12[2 * n + 1];
        dx = I.kx * rt[0] * (I.A * ct[0] + e1 * ct[1]);
        dy = I.ky * rt[1] * (I.A * ct[2] + e2 * ct[3]);
      } else {
        dx = I.cdx;
        dy = I.cdy;
      }
      const T nlo_y = T(-k), nhi_y = T(ny - 1 - k), nlo_x = T(-i), nhi_x = T(nx - 1 - i);
      int64_t rq[Q];
      T w0[Q], w1[Q], w2[Q], w3[Q];
      T exit_y = T(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T d = dy + I.gy[q];
        const bool out = (d < nlo_y) || (d > nhi_y);
        const T fl = floor(d);
        int c = k + (int)fl;
        T tt = d - fl;
        if (c > ny - 2) {
          c = ny - 2;
          tt = T(1);
        }
        if (!out && (c < 0)) bad |= 1u;
        const T wq = out ? T(0) : I.w[q];
        exit_y += I.w[q] - wq;
        rq[q] = out ? (int64_t)k * nx : (int64_t)c * nx;
        const T t2 = tt * tt, omt = T(1) - tt;
        w0[q] = wq;
        w1[q] = wq * (t2 * (T(3) - T(2) * tt));
        w2[q] = wq * (tt * omt * omt);
        w3[q] = -wq * (t2 * omt);
      }
      const T om = T(1) - uj;
      T acc = T(0);
#pragma unroll 1
      for (int p = 0; p < Q; ++p) {
        const T d = dx + I.gx[p];
        if ((d < nlo_x) || (d > nhi_x)) {
          acc += I.w[p] * om;
          continue;
        }
        const T fl = floor(d);
        int c = i + (int)fl;
        T tt = d - fl;
        if (c > nx - 2) {
          c = nx - 2;
          tt = T(1);
        }
        const T t2 = tt * tt, omt = T(1) - tt;
        const T h01 = t2 * (T(3) - T(2) * tt), h10 = tt * omt * omt, h11 = -(t2 * omt);
        T accp = exit_y * om;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int64_t o = rq[q] + c;
          const V4<T> r0 = R[o];
          const V4<T> r1 = R[o + nx];
          const V2<T> s0 = S[o];
          const V2<T> s1 = S[o + nx];
          const T a0 = (r0.x - uj) + h01 * r0.y + h10 * r0.z + h11 * r0.w;
          const T a1 = (r1.x - uj) + h01 * r1.y + h10 * r1.z + h11 * r1.w;
          const T b0 = s0.x + h01 * s0.y;
          const T b1 = s1.x + h01 * s1.y;
          accp += w0[q] * a0;
          accp += w1[q] * (a1 - a0);
          accp += w2[q] * b0;
          accp += w3[q] * b1;
        }
        acc += I.w[p] * accp;
      }
      T* dst = I.buf[(n_steps - m) & 1];
      dst[jn] = uj + acc;
      const bool L = (i == 1), Rt = (i == nx - 2), B = (k == 1), Tp = (k == ny - 2);
      if (L | Rt | B | Tp) {
        const int64_t top = (int64_t)(ny - 1) * nx, rw = (int64_t)k * nx;
        if (L) dst[rw] = T(1);
        if (Rt) dst[rw + nx - 1] = T(1);
        if (B) dst[i] = T(1);
        if (Tp) dst[top + i] = T(1);
        if (L & B) dst[0] = T(1);
        if (Rt & B) dst[nx - 1] = T(1);
        if (L & Tp) dst[top] = T(1);
        if (Rt & Tp) dst[top + nx - 1] = T(1);
      }
    }
    if (!grid_barrier(bar, expected, err)) return;
  }
  if (bad) atomicOr(err, FK_DEVERR_RANGE);
}

// ------------------------------------------------------------------ host --

const int kSideStreams = 8;  // the default number of hardware work queues

enum { kModeNone = 0, kModePersistent = 1, kModeStreams = 2 };

struct BatchWork {
  void* d_inst = nullptr;  // instance table (device copy)
  size_t d_inst_bytes = 0;
  void* d_e12 = nullptr;   // per-instance per-step drift scalars
  size_t d_e12_bytes = 0;
  BarrierState* d_bar = nullptr;
  // one cached graph: key = (plans, inputs, outputs, grid)
  std::vector<const void*> key;
  cudaGraphExec_t graph = nullptr;
  // concurrent single-plan strategy: side streams and fork/join events
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork = nullptr, join[kSideStreams] = {};
  int mode = kModeNone;  // strategy of the last call
};

std::mutex g_batch_mu;

struct BatchTune {
  int n_inst, q, elem, n_steps;
  int64_t nodes;
  int blocks_per_sm;
  int mode;
};
std::vector<BatchTune> g_batch_tune;

template <typename T, int Q>
cudaError_t launch_batched(const BInst<T>* d_inst, int n_inst, int n_steps, int total_r,
                           int total_q, unsigned expected, BarrierState* bar, unsigned* err,
                           int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batched<T, Q>, d_inst, n_inst, n_steps, total_r, total_q,
                            expected, bar, err);
}

template <typename T>
cudaError_t launch_q(int q, const BInst<T>* d_inst, int n_inst, int n_steps, int total_r,
                     int total_q, unsigned expected, BarrierState* bar, unsigned* err, int grid,
                     cudaStream_t s) {
  switch (q) {
#define FK_CASE(QQ)                                                                     \
  case QQ:                                                                              \
    return launch_batched<T, QQ>(d_inst, n_inst, n_steps, total_r, total_q, expected, bar, \
                                 err, grid, s);
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
#undef FK_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
int max_blocks_per_sm(int q) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (q) {
#define FK_CASE(QQ) \
  case QQ: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<T, QQ>, 256, 0); break;
    FK_CASE(1) FK_CASE(2) FK_CASE(3) FK_CASE(4) FK_CASE(5) FK_CASE(6) FK_CASE(7) FK_CASE(8)
#undef FK_CASE
    default: break;
  }
  return e == cudaSuccess ? nb : 0;
}

fk_status grow(fk_plan* p, void** ptr, size_t* have, size_t need) {
  if (*have >= need) return FK_OK;
  fk_dev_free(*ptr);
  *ptr = nullptr;
  *have = 0;
  fk_status st = fk_dev_alloc(p, ptr, need);
  if (st == FK_OK) *have = need;
  return st;
}

// Input staging of one instance (same rule as the single-plan march): the
// buffer that step 1 reads must not be the one it writes.
template <typename T>
cudaError_t stage_input(fk_plan* p, const void* u_terminal, void* u_out, int N, const T** first,
                        cudaStream_t s) {
  const bool first_to_out = ((N - 1) % 2) == 0;
  const void* src = u_terminal;
  cudaError_t e = cudaSuccess;
  if (!src) {
    void* buf = first_to_out ? p->scratch : u_out;
    e = fk_launch_fill_chi(buf, 2, p->grid.n[0], p->grid.n[1], (int)sizeof(T), s);
    src = buf;
  } else if (src == u_out && first_to_out) {
    e = fk_launch_copy(p->scratch, src, p->J * (int64_t)sizeof(T), s);
    src = p->scratch;
  }
  *first = (const T*)src;
  return e;
}

fk_status ensure_side_streams(BatchWork* bw) {
  if (bw->fork) return FK_OK;
  if (cudaEventCreateWithFlags(&bw->fork, cudaEventDisableTiming) != cudaSuccess) return FK_ERR_CUDA;
  for (int k = 0; k < kSideStreams; ++k) {
    if (cudaStreamCreateWithFlags(&bw->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bw->join[k], cudaEventDisableTiming) != cudaSuccess)
      return FK_ERR_CUDA;
  }
  return FK_OK;
}

// Largest instances first, each on the side stream with the least work so
// far (longest-processing-time order).
std::vector<int> assign_streams(int n, fk_plan* const* plans, int K) {
  std::vector<int> order(n), which(n);
  for (int b = 0; b < n; ++b) order[b] = b;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return plans[x]->J > plans[y]->J; });
  std::vector<int64_t> load(K, 0);
  for (int b : order) {
    int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    which[b] = k;
    load[k] += plans[b]->J;
  }
  return which;
}

// Steps n_from-1 .. n_to of every instance (the whole march when n_from =
// N and n_to = 0, through each plan's graph; otherwise direct launches) on
// the side streams, between a fork and a join on `stream`.
fk_status run_streams(int n, fk_plan* const* plans, const void* const* u_terminal,
                      void* const* u_out, int n_from, int n_to, cudaStream_t stream,
                      BatchWork* bw) {
  fk_status st = ensure_side_streams(bw);
  if (st != FK_OK) return st;
  const int K = n < kSideStreams ? n : kSideStreams;
  const std::vector<int> which = assign_streams(n, plans, K);
  if (cudaEventRecord(bw->fork, stream) != cudaSuccess) return FK_ERR_CUDA;
  for (int k = 0; k < K; ++k)
    if (cudaStreamWaitEvent(bw->side[k], bw->fork, 0) != cudaSuccess) return FK_ERR_CUDA;
  const bool whole = n_from == plans[0]->n_steps && n_to == 0;
  for (int b = 0; b < n && st == FK_OK; ++b) {
    cudaStream_t sb = bw->side[which[b]];
    // no persistent march here: its CTAs wait on one another, which the
    // plans running concurrently on other streams must not stand in for
    plans[b]->no_persist = 1;
    st = whole ? fk_solve(plans[b], u_terminal[b], u_out[b], nullptr, 0, sb)
               : fk_march(plans[b], n_from, n_to, u_terminal[b], u_out[b], sb);
    plans[b]->no_persist = 0;
  }
  // join every side stream, also after a failed enqueue
  for (int k = 0; k < K; ++k) {
    if (cudaEventRecord(bw->join[k], bw->side[k]) != cudaSuccess ||
        cudaStreamWaitEvent(stream, bw->join[k], 0) != cudaSuccess)
      return FK_ERR_CUDA;
  }
  return st;
}

template <typename T>
fk_status run_batch(int n, fk_plan* const* plans, const void* const* u_terminal, void* const* u_out,
                    cudaStream_t stream) {
  fk_plan* p0 = plans[0];
  const int q = p0->q, N = p0->n_steps;
  std::vector<BInst<T>> inst(n);
  std::vector<T> e12((size_t)n * N * 2);
  int total_r = 0, total_q = 0;
  int64_t nodes = 0;
  bool aliased = false;
  for (int b = 0; b < n; ++b) {
    fk_plan* p = plans[b];
    if (!p->batch_rec) {
      fk_status st = fk_dev_alloc(p, &p->batch_rec, (size_t)p->J * 6 * sizeof(T));
      if (st != FK_OK) return st;
    }
    BInst<T>& I = inst[b];
    memset(&I, 0, sizeof(I));
    I.nx = p->grid.n[0];
    I.ny = p->grid.n[1];
    I.family = p->coeffs.family;
    I.rec = (V4<T>*)p->batch_rec;
    I.srec = (V2<T>*)((char*)p->batch_rec + (size_t)p->J * 4 * sizeof(T));
    I.col_tab = (const T*)p->col_tab;
    I.row_tab = (const T*)p->row_tab;
    I.tiles_x_all = (I.nx - 1 + kTileW - 1) / kTileW;
    I.tiles_all = I.tiles_x_all * ((I.ny + kTileH - 1) / kTileH);
    I.tiles_x_int = (I.nx - 2 + kTileW - 1) / kTileW;
    I.tiles_int = I.tiles_x_int * ((I.ny - 2 + kTileH - 1) / kTileH);
    I.first_r = total_r;
    I.first_q = total_q;
    total_r += I.tiles_all;
    total_q += I.tiles_int;
    nodes += p->J;
    // the same per-axis factors and per-step scalars as the single-plan kernel
    for (int s = 0; s < N; ++s) {
      Step2D<T> a;
      if (sizeof(T) == 4)
        fk_fill_step2d_f32(p, s, (Step2D<float>*)&a);
      else
        fk_fill_step2d_f64(p, s, (Step2D<double>*)&a);
      e12[((size_t)b * N + s) * 2] = a.e1;
      e12[((size_t)b * N + s) * 2 + 1] = a.e2;
      if (s == 0) {
        I.kx = a.kx;
        I.ky = a.ky;
        I.A = a.A;
        I.cdx = a.cdx;
        I.cdy = a.cdy;
        for (int m = 0; m < q; ++m) {
          I.gx[m] = a.gx[m];
          I.gy[m] = a.gy[m];
          I.w[m] = a.w[m];
        }
      }
    }
    I.buf[0] = (T*)u_out[b];  // step m writes buf[(N - m) & 1]
    I.buf[1] = (T*)p->scratch;
    if (u_terminal[b] && u_terminal[b] == u_out[b]) aliased = true;
  }
  BatchWork* bw = (BatchWork*)p0->batch_work;
  if (!bw) {
    bw = new BatchWork();
    p0->batch_work = bw;
  }
  // the persistent kernel knows uniform meshes of boxes whose faces all
  // absorb and the two families of its own step; other batches run the
  // plans' own graphs
  for (int b = 0; b < n; ++b) {
    if (plans[b]->periodic_x || plans[b]->nu || plans[b]->coeffs.family == FK_PAPER_CELLULAR) {
      bw->mode = kModeStreams;
      p0->batch_grid = 0;
      return run_streams(n, plans, u_terminal, u_out, N, 0, stream, bw);
    }
  }
  fk_status st = grow(p0, &bw->d_inst, &bw->d_inst_bytes, sizeof(BInst<T>) * n);
  if (st == FK_OK) st = grow(p0, &bw->d_e12, &bw->d_e12_bytes, sizeof(T) * e12.size());
  if (st == FK_OK && !bw->d_bar) st = fk_dev_alloc(p0, (void**)&bw->d_bar, sizeof(BarrierState));
  if (st != FK_OK) return st;
  for (int b = 0; b < n; ++b) inst[b].e12 = (const T*)bw->d_e12 + (size_t)b * N * 2;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return FK_ERR_CUDA;
  if (cudaMemcpy(bw->d_e12, e12.data(), sizeof(T) * e12.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return FK_ERR_CUDA;

  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p0->device);
  const int max_bps = max_blocks_per_sm<T>(q);
  if (max_bps < 1 || sms < 1) return FK_ERR_UNSUPPORTED;
  // ---- autotune the CTAs per SM once per batch shape (on chi-filled
  // buffers, before the real inputs are staged; skipped when an input
  // aliases its output)
  int bps = max_bps;
  // without a timing: the persistent kernel for small instances
  int mode = nodes / n < 16384 ? kModePersistent : kModeStreams;
  // explicit CTAs per SM (profiling runs, where timing is distorted)
  const char* fixed = getenv("FK_BATCH_CTAS_PER_SM");
  if (fixed && atoi(fixed) >= 1 && atoi(fixed) <= max_bps) {
    bps = atoi(fixed);
    mode = kModePersistent;
  } else {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    bool found = false;
    for (const BatchTune& t : g_batch_tune)
      if (t.n_inst == n && t.q == q && t.elem == (int)sizeof(T) && t.n_steps == N &&
          t.nodes == nodes) {
        bps = t.blocks_per_sm;
        mode = t.mode;
        found = true;
      }
    if (!found && !aliased) {
      std::vector<BInst<T>> tune = inst;
      for (int b = 0; b < n; ++b) {
        fk_launch_fill_chi(tune[b].buf[0], 2, tune[b].nx, tune[b].ny, (int)sizeof(T), stream);
        fk_launch_fill_chi(tune[b].buf[1], 2, tune[b].nx, tune[b].ny, (int)sizeof(T), stream);
        tune[b].u_first = tune[b].buf[1];
      }
      cudaStreamSynchronize(stream);
      cudaMemcpy(bw->d_inst, tune.data(), sizeof(BInst<T>) * n, cudaMemcpyHostToDevice);
      const int steps = N < 4 ? N : 4;
      float best = 1e30f;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      const bool log = getenv("FK_TUNE_LOG") != nullptr;
      for (int cand = max_bps; cand >= 1; --cand) {
        cudaMemsetAsync(bw->d_bar, 0, sizeof(BarrierState), stream);
        cudaEventRecord(e0, stream);
        cudaError_t e = launch_q<T>(q, (const BInst<T>*)bw->d_inst, n, steps, total_r, total_q,
                                    (unsigned)(sms * cand), bw->d_bar, p0->d_err, sms * cand,
                                    stream);
        cudaEventRecord(e1, stream);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (log)
          fprintf(stderr, "fk batched autotune: %d CTAs/SM  %.3f ms / %d steps\n", cand, ms, steps);
        if (ms < best) {
          best = ms;
          bps = cand;
        }
      }
      mode = kModePersistent;
      // the concurrent single-plan marches over the same steps, from chi
      // in the output buffers (which no input aliases here)
      for (int b = 0; b < n; ++b)
        fk_launch_fill_chi(u_out[b], 2, plans[b]->grid.n[0], plans[b]->grid.n[1], (int)sizeof(T),
                           stream);
      std::vector<const void*> ins(u_out, u_out + n);
      cudaEventRecord(e0, stream);
      fk_status ss = run_streams(n, plans, ins.data(), u_out, N, N - steps, stream, bw);
      cudaEventRecord(e1, stream);
      if (ss == FK_OK && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (log) fprintf(stderr, "fk batched autotune: concurrent plans  %.3f ms / %d steps\n", ms, steps);
        if (ms < best) mode = kModeStreams;
      }
      cudaGetLastError();
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaStreamSynchronize(stream);
      cudaMemset(p0->d_err, 0, sizeof(unsigned));
      for (int b = 0; b < n; ++b) cudaMemset(plans[b]->d_err, 0, sizeof(unsigned));
      g_batch_tune.push_back({n, q, (int)sizeof(T), N, nodes, bps, mode});
      bw->key.clear();  // the device table now holds the tuning copy
    }
  }
  // explicit strategy (tests): FK_BATCH_MODE=persistent|streams
  if (const char* m = getenv("FK_BATCH_MODE")) {
    if (strcmp(m, "persistent") == 0) mode = kModePersistent;
    if (strcmp(m, "streams") == 0) mode = kModeStreams;
  }
  bw->mode = mode;
  if (mode == kModeStreams) {
    p0->batch_grid = 0;
    return run_streams(n, plans, u_terminal, u_out, N, 0, stream, bw);
  }
  const int grid = sms * bps;
  // test hook: one phantom CTA that never arrives makes every barrier wait
  // run into its limit, which exercises the timeout path
  const unsigned expected = (unsigned)grid + (getenv("FK_TEST_STALL_BARRIER") ? 1u : 0u);
  std::vector<const void*> key;
  key.reserve(3 * n + 2);
  for (int b = 0; b < n; ++b) {
    key.push_back(plans[b]);
    key.push_back(u_terminal[b]);
    key.push_back(u_out[b]);
  }
  key.push_back((const void*)(intptr_t)grid);
  key.push_back((const void*)(intptr_t)expected);
  if (key != bw->key || !bw->graph) {
    if (bw->graph) {
      cudaGraphExecDestroy(bw->graph);
      bw->graph = nullptr;
    }
    bw->key.clear();
    // instance table: inputs as they will be staged inside the graph
    for (int b = 0; b < n; ++b) {
      const bool first_to_out = ((N - 1) % 2) == 0;
      const void* src = u_terminal[b];
      if (!src)
        src = first_to_out ? plans[b]->scratch : u_out[b];
      else if (src == u_out[b] && first_to_out)
        src = plans[b]->scratch;
      inst[b].u_first = (const T*)src;
    }
    if (cudaMemcpy(bw->d_inst, inst.data(), sizeof(BInst<T>) * n, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return FK_ERR_CUDA;
    cudaStream_t cs = p0->cap_stream;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return FK_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < n && e == cudaSuccess; ++b) {
      const T* first;
      e = stage_input<T>(plans[b], u_terminal[b], u_out[b], N, &first, cs);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(bw->d_bar, 0, sizeof(BarrierState), cs);
    if (e == cudaSuccess)
      e = launch_q<T>(q, (const BInst<T>*)bw->d_inst, n, N, total_r, total_q, expected, bw->d_bar,
                      p0->d_err, grid, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bw->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bw->graph = nullptr;
      return FK_ERR_CUDA;
    }
    bw->key = key;
  }
  p0->batch_grid = grid;
  return cudaGraphLaunch(bw->graph, stream) == cudaSuccess ? FK_OK : FK_ERR_CUDA;
}

}  // namespace

int fk_batch_mode(const fk_plan* p) {
  const BatchWork* bw = (const BatchWork*)p->batch_work;
  return bw ? bw->mode : kModeNone;
}

void fk_batch_release(fk_plan* p) {
  BatchWork* bw = (BatchWork*)p->batch_work;
  if (!bw) return;
  if (bw->graph) cudaGraphExecDestroy(bw->graph);
  for (int k = 0; k < kSideStreams; ++k) {
    if (bw->side[k]) cudaStreamDestroy(bw->side[k]);
    if (bw->join[k]) cudaEventDestroy(bw->join[k]);
  }
  if (bw->fork) cudaEventDestroy(bw->fork);
  fk_dev_free(bw->d_inst);
  fk_dev_free(bw->d_e12);
  fk_dev_free(bw->d_bar);
  delete bw;
  p->batch_work = nullptr;
}

extern "C" fk_status fk_solve_batched(int n, fk_plan* const* plans, const void* const* u_terminal,
                                      void* const* u_out, cudaStream_t stream) {
  FkRange range("fk_solve_batched");
  if (n < 1 || n > kMaxInst || !plans || !u_terminal || !u_out) return FK_ERR_INVALID_ARG;
  for (int b = 0; b < n; ++b) {
    if (!plans[b] || !u_out[b]) return FK_ERR_INVALID_ARG;
    const fk_plan* p = plans[b];
    if (p->grid.dim != 2 || p->path != FK_PATH_MATRIX_FREE) return FK_ERR_UNSUPPORTED;
    if (p->prec != plans[0]->prec || p->q != plans[0]->q || p->n_steps != plans[0]->n_steps ||
        p->device != plans[0]->device)
      return FK_ERR_UNSUPPORTED;
    for (int c = 0; c < b; ++c)
      if (plans[c] == p || u_out[c] == u_out[b]) return FK_ERR_INVALID_ARG;
  }
  return plans[0]->prec == FK_FP32 ? run_batch<float>(n, plans, u_terminal, u_out, stream)
                                   : run_batch<double>(n, plans, u_terminal, u_out, stream);
}
