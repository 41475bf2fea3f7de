// fk_solve_static: the 2D matrix-free march with no device allocation.
//
// Some callers cannot call cudaMalloc: applications that hand every byte of
// device memory to their own pool allocator and forbid libraries from
// allocating beside it, and latency-bound loops that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree.  For them this
// entry point keeps everything the march needs besides the caller's input
// and output -- the ping-pong field, the per-row and per-column coefficient
// tables and the device error word -- in one file-scope __device__ array of
// FK_STATIC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  fk_static_last_device_error reads the error
// word back (it synchronises the device, so it is for after the work).
//
// The step kernel is the same one fk_solve launches; only where its
// scratch lives differs.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "fk_internal.h"

#define FK_STATIC_SCRATCH_BYTES (16u << 20)  // 16 MiB
#define FK_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char fk_static_scratch[FK_STATIC_SCRATCH_BYTES];

namespace {

const double kPi = 3.14159265358979323846264338327950288;

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[FK_STATIC_MAX_DEVICES];  // device address of the array, per device

// Per-column sin(pi x), sin(2 pi x), cos(pi x), cos(2 pi x) and per-row
// cos(pi y), sin(pi y), evaluated in double like the plan's host tables.
template <typename T>
__global__ void k_static_tables(T* col, T* row, int nx, int ny, double lox, double hx,
                                double loy, double hy) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nx) {
    const double x = lox + t * hx;
    col[4 * t + 0] = (T)sin(kPi * x);
    col[4 * t + 1] = (T)sin(2.0 * kPi * x);
    col[4 * t + 2] = (T)cos(kPi * x);
    col[4 * t + 3] = (T)cos(2.0 * kPi * x);
  }
  if (t < ny) {
    const double y = loy + t * hy;
    row[2 * t + 0] = (T)cos(kPi * y);
    row[2 * t + 1] = (T)sin(kPi * y);
  }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Once per device, with that device current: the device address of the
// static array (its host-side name is only a stand-in) and the opt-in to
// large dynamic shared memory of every step kernel this entry can launch.
fk_status setup_device(int dev, unsigned char** addr) {
  if (dev < 0 || dev >= FK_STATIC_MAX_DEVICES) return FK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, fk_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FK_ERR_CUDA;
    }
    for (int q = 1; q <= FK_MAXQ_2D; ++q) {
      if (fk_prepare_step_kernels(2, q, 4) != cudaSuccess ||
          fk_prepare_step_kernels(2, q, 8) != cudaSuccess) {
        cudaGetLastError();
        return FK_ERR_CUDA;
      }
    }
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *addr = g_scratch_addr[dev];
  return FK_OK;
}

bool finite_d(double v) { return v == v && v - v == 0.0; }

}  // namespace

extern "C" fk_status fk_solve_static(const fk_grid* grid, const fk_coeffs* coeffs, int q_per_dim,
                                     double dt, int n_steps, fk_precision prec,
                                     const void* u_terminal, void* u_out, cudaStream_t stream) {
  // ---- arguments (no CUDA call before they are checked)
  if (!grid || !coeffs || !u_out) return FK_ERR_INVALID_ARG;
  if (grid->dim != 2) return FK_ERR_UNSUPPORTED;
  if (grid->axis[0] || grid->axis[1]) return FK_ERR_UNSUPPORTED;  // uniform meshes only
  for (int m = 0; m < 2; ++m) {
    if (grid->n[m] < 3 || !finite_d(grid->lo[m]) || !finite_d(grid->hi[m]) ||
        !(grid->hi[m] > grid->lo[m]))
      return FK_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !finite_d(dt) || n_steps < 1) return FK_ERR_INVALID_ARG;
  if (prec != FK_FP32 && prec != FK_FP64) return FK_ERR_INVALID_ARG;
  if (coeffs->family != FK_CONST_DRIFT && coeffs->family != FK_CELLULAR_FLOW)
    return FK_ERR_INVALID_ARG;
  for (int k = 0; k < 16; ++k)
    if (!finite_d(coeffs->p[k])) return FK_ERR_INVALID_ARG;
  if (!(coeffs->p[3] >= 0.0)) return FK_ERR_INVALID_ARG;
  if (q_per_dim < 1 || q_per_dim > FK_MAXQ_2D) return FK_ERR_UNSUPPORTED;

  // ---- a plan description on the stack (the plan object owns no memory here)
  fk_plan p;
  memset(&p, 0, sizeof(p));
  p.grid = *grid;
  p.grid.n[2] = 1;
  p.coeffs = *coeffs;
  p.q = q_per_dim;
  p.dt = dt;
  p.n_steps = n_steps;
  p.prec = prec;
  p.path = FK_PATH_MATRIX_FREE;
  p.elem = prec == FK_FP32 ? 4 : 8;
  if (fk_gauss_hermite(q_per_dim, p.gh_a, p.gh_w) != FK_OK) return FK_ERR_INVALID_ARG;
  const int nx = grid->n[0], ny = grid->n[1];
  p.J = (int64_t)nx * ny;
  for (int m = 0; m < 2; ++m) p.h[m] = (grid->hi[m] - grid->lo[m]) / (grid->n[m] - 1);
  const double sg = (coeffs->family == FK_CONST_DRIFT ? coeffs->p[3] : sqrt(2.0 * coeffs->p[3])) *
                    sqrt(2.0 * dt);
  double bmax[2];
  if (coeffs->family == FK_CONST_DRIFT) {
    bmax[0] = fabs(coeffs->p[0]);
    bmax[1] = fabs(coeffs->p[1]);
  } else {
    bmax[0] = kPi * (fabs(coeffs->p[0]) + fabs(coeffs->p[1]));
    bmax[1] = kPi * (fabs(coeffs->p[0]) + 2.0 * fabs(coeffs->p[1]));
  }
  for (int m = 0; m < 2; ++m) {
    p.reach[m] = (bmax[m] * dt + sg * fabs(p.gh_a[0])) / p.h[m];
    const double r = p.reach[m] * (1.0 + 1e-6) + 1e-3;
    if (r > 4096.0) return FK_ERR_UNSUPPORTED;
    p.halo[m] = (int)ceil(r) + 1;
  }
  // ---- the static array must hold the error word, both tables and one field
  const size_t off_col = 256;
  const size_t off_row = align256(off_col + (size_t)4 * nx * p.elem);
  const size_t off_fld = align256(off_row + (size_t)2 * ny * p.elem);
  const size_t need = off_fld + (size_t)p.J * p.elem;
  if (need > FK_STATIC_SCRATCH_BYTES) return FK_ERR_INVALID_ARG;

  // ---- a CUDA error left pending by the caller's earlier work is not ours
  // to clear or to blame on this call's launches: report it, enqueue nothing
  if (cudaPeekAtLastError() != cudaSuccess) return FK_ERR_CUDA;

  // ---- device set-up (first call on each device) and tile choice
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FK_ERR_CUDA;
  unsigned char* base = nullptr;
  fk_status st = setup_device(dev, &base);
  if (st != FK_OK) return st;
  int smem_max = 0;
  if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return FK_ERR_CUDA;
  static const int tiles[][2] = {{32, 16}, {32, 8}, {32, 4}};
  bool fits = false;
  for (int c = 0; c < 3 && !fits; ++c) {
    const int lx = tiles[c][0] + 2 * p.halo[0] + 2, ly = tiles[c][1] + 2 * p.halo[1] + 2;
    if (fk_step2d_smem(lx, ly, ly | 1, p.elem) <= (size_t)smem_max) {
      p.tile[0] = tiles[c][0];
      p.tile[1] = tiles[c][1];
      fits = true;
    }
  }
  if (!fits) return FK_ERR_UNSUPPORTED;
  p.d_err = (unsigned*)base;
  p.col_tab = base + off_col;
  p.row_tab = base + off_row;
  p.scratch = base + off_fld;

  // ---- enqueue: clear the error word, tables, then the ping-pong march
  // (the last step lands in u_out; u_terminal is only read)
  if (cudaMemsetAsync(p.d_err, 0, sizeof(unsigned), stream) != cudaSuccess) return FK_ERR_CUDA;
  const int tb = 256, nb = ((nx > ny ? nx : ny) + tb - 1) / tb;
  if (prec == FK_FP32)
    k_static_tables<float><<<nb, tb, 0, stream>>>((float*)p.col_tab, (float*)p.row_tab, nx, ny,
                                                  grid->lo[0], p.h[0], grid->lo[1], p.h[1]);
  else
    k_static_tables<double><<<nb, tb, 0, stream>>>((double*)p.col_tab, (double*)p.row_tab, nx, ny,
                                                   grid->lo[0], p.h[0], grid->lo[1], p.h[1]);
  if (cudaGetLastError() != cudaSuccess) return FK_ERR_CUDA;
  const int64_t bytes = p.J * p.elem;
  const bool first_to_out = ((n_steps - 1) % 2) == 0;
  const void* src = u_terminal;
  if (!src) {
    void* buf = first_to_out ? p.scratch : u_out;
    if (fk_launch_fill_chi(buf, 2, nx, ny, p.elem, stream) != cudaSuccess) return FK_ERR_CUDA;
    src = buf;
  } else if (src == u_out && first_to_out) {
    if (fk_launch_copy(p.scratch, src, bytes, stream) != cudaSuccess) return FK_ERR_CUDA;
    src = p.scratch;
  }
  for (int m = 1; m <= n_steps; ++m) {
    const int n = n_steps - m;
    void* dst = ((n_steps - m) % 2 == 0) ? u_out : p.scratch;
    cudaError_t e;
    if (prec == FK_FP32) {
      Step2D<float> a;
      fk_fill_step2d_f32(&p, n, &a);
      a.u_in = (const float*)src;
      a.u_out = (float*)dst;
      a.snap = nullptr;
      e = fk_launch_step2d<float>(a, q_per_dim, stream);
    } else {
      Step2D<double> a;
      fk_fill_step2d_f64(&p, n, &a);
      a.u_in = (const double*)src;
      a.u_out = (double*)dst;
      a.snap = nullptr;
      e = fk_launch_step2d<double>(a, q_per_dim, stream);
    }
    if (e != cudaSuccess) return FK_ERR_CUDA;
    src = dst;
  }
  return FK_OK;
}

extern "C" fk_status fk_static_last_device_error(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FK_ERR_CUDA;
  unsigned char* base = nullptr;
  fk_status st = setup_device(dev, &base);
  if (st != FK_OK) return st;
  // the calls are asynchronous on the caller's streams, which need not
  // synchronise with the legacy default stream: wait for the whole device
  if (cudaDeviceSynchronize() != cudaSuccess) return FK_ERR_CUDA;
  unsigned word = 0;
  const unsigned zero = 0;
  if (cudaMemcpy(&word, base, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(base, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
    return FK_ERR_CUDA;
  if (word & FK_DEVERR_TIMEOUT) return FK_ERR_TIMEOUT;
  return word ? FK_ERR_DEVICE : FK_OK;
}
