// Plan object, argument validation, Gauss-Hermite rule and the march driver
// of the C ABI (include/fk.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <iterator>
#include <mutex>
#include <new>
#include <vector>

#include "fk_internal.h"

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------- quadrature --
// Polynomials orthonormal for the probability density pi^{-1/2} exp(-x^2)
// satisfy x p_k = b_{k+1} p_{k+1} + b_k p_{k-1} with b_k = sqrt(k/2),
// p_0 = 1.  The Gauss nodes are the zeros of p_q; they are bracketed by a
// sign scan over (-sqrt(2q+1), sqrt(2q+1)) (a bound on the zeros of the
// Hermite polynomials) and refined by bisection to the last bit.  The
// weight of node x is the Christoffel number 1 / sum_{k<q} p_k(x)^2, so the
// weights of the probability measure sum to 1 (Eq. (expec)).
double orthonormal_hermite(int q, double x, double* sum_sq) {
  double pm = 0.0, p = 1.0, s = 1.0;
  for (int k = 0; k < q; ++k) {
    const double bk = sqrt(0.5 * k), bk1 = sqrt(0.5 * (k + 1));
    const double pn = (x * p - bk * pm) / bk1;
    pm = p;
    p = pn;
    if (k + 1 < q) s += p * p;
  }
  if (sum_sq) *sum_sq = s;
  return p;
}

bool gauss_hermite(int q, double* a, double* w) {
  if (q < 1 || q > FK_MAXQ) return false;
  const double lim = sqrt(2.0 * q + 1.0);
  const int scan = 4000 * q;
  int found = 0;
  double xl = -lim, fl = orthonormal_hermite(q, xl, nullptr);
  for (int s = 1; s <= scan && found < q; ++s) {
    const double xr = -lim + 2.0 * lim * s / scan;
    const double fr = orthonormal_hermite(q, xr, nullptr);
    if (fr == 0.0) {
      a[found++] = xr;
    } else if ((fl < 0.0) != (fr < 0.0) && fl != 0.0) {
      double lo = xl, hi = xr, flo = fl;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = orthonormal_hermite(q, mid, nullptr);
        if (fm == 0.0) {
          lo = hi = mid;
          break;
        }
        if ((fm < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      a[found++] = 0.5 * (lo + hi);
    }
    xl = xr;
    fl = fr;
  }
  if (found != q) return false;
  // symmetrise (the rule is symmetric about 0)
  for (int i = 0; i < q / 2; ++i) {
    const double m = 0.5 * (a[q - 1 - i] - a[i]);
    a[i] = -m;
    a[q - 1 - i] = m;
  }
  if (q % 2) a[q / 2] = 0.0;
  double tot = 0.0;
  for (int i = 0; i < q; ++i) {
    double s;
    orthonormal_hermite(q, a[i], &s);
    w[i] = 1.0 / s;
    tot += w[i];
  }
  (void)tot;
  return true;
}

bool finite(double v) { return v == v && v - v == 0.0; }

// Largest |b| over the box (drift bound used to size the tile halo).
void drift_bound(const fk_coeffs* c, int dim, double* bmax) {
  for (int m = 0; m < 3; ++m) bmax[m] = 0.0;
  if (c->family == FK_RUNAWAY_3D || c->family == FK_RUNAWAY_QUENCH_3D)
    return;  // per-node bounds: runaway_bounds()
  if (c->family == FK_CONST_DRIFT) {
    for (int m = 0; m < dim; ++m) bmax[m] = fabs(c->p[m]);
  } else if (c->family == FK_PAPER_CELLULAR) {
    const double Pe = fabs(c->p[0]), n = fabs(c->p[1]), e = fabs(c->p[2]);
    bmax[0] = Pe * kPi * (1.0 + e);
    bmax[1] = Pe * n * (1.0 + e);
  } else {
    const double A = fabs(c->p[0]), e = fabs(c->p[1]);
    bmax[0] = kPi * (A + e);
    bmax[1] = kPi * (A + 2.0 * e);
  }
}

double sigma_of(const fk_coeffs* c) {
  if (c->family == FK_PAPER_CELLULAR) return 1.0;  // unit Brownian motions
  if (c->family == FK_RUNAWAY_3D || c->family == FK_RUNAWAY_QUENCH_3D)
    return 0.0;  // per node: runaway_bounds()
  return c->family == FK_CONST_DRIFT ? c->p[3] : sqrt(2.0 * c->p[3]);
}

// Drift and diagonal sigma of the runaway-electron model at one node (the
// host's copy of Eq. (ex32d), for the plan's window bounds only).
void runaway_host(const double* q, double mom, double xi, double r, double* b, double* s) {
  const double E = q[0], tau = q[1], Z = q[2], delta = q[3], nu = q[4], vT = q[5];
  const double rD = q[6], Wr = q[7], Dp = q[8], V0 = q[9], D0 = q[10];
  const double gam = sqrt(1.0 + (delta * mom) * (delta * mom)), y = mom / gam;
  const double phi = erf(y), dphi = 2.0 / sqrt(kPi) * exp(-y * y);
  const double psi = (phi - y * dphi) / (2.0 * y * y), dpsi = dphi - 2.0 * psi / y;
  const double nv2 = nu * vT * vT;
  const double CA = nv2 * psi / y;
  const double CB = 0.5 * nv2 / y * (Z + phi - psi + 0.5 * y * y * pow(delta, 4.0));
  const double CF = 2.0 * nu * vT * psi;
  const double df = 2.0 * mom * psi / y +
                    mom * mom * (dpsi / y - psi / (y * y)) / (gam * gam * gam);
  const double om = 1.0 - xi * xi;
  b[0] = E * xi - gam * mom / tau * om - CF + nv2 * df / (mom * mom);
  b[1] = E * om / mom - xi * om / (tau * gam) - 2.0 * xi * CB / (mom * mom);
  const double th = tanh((r - rD) / Wr), ep = exp(-(mom / Dp) * (mom / Dp));
  b[2] = (r > rD ? V0 : 0.0) + 0.5 * D0 * (1.0 - th * th) / Wr * ep;
  s[0] = sqrt(2.0 * CA);
  s[1] = sqrt(2.0 * CB) * sqrt(om > 0.0 ? om : 0.0) / mom;
  s[2] = sqrt(D0 * (1.0 + th) * ep);
}

// The thermal-quench schedule (end of Sec. 4.3): the static runaway
// constants at time t (see fk_runaway_quench_params in fk.h).
void quench_params(const double* q, double t, double* p11) {
  const double T = q[4] + (q[3] - q[4]) * exp(-t / q[6]);
  const double c = 14.9 - 0.5 * log(0.28);
  const double lam = c + log(T), lam_ref = c + log(q[5]);
  p11[0] = q[0] * pow(q[3] / T, 1.5);
  p11[1] = q[1];
  p11[2] = q[2];
  p11[3] = sqrt(2.0 * T / q[12]);
  p11[4] = pow(q[5] / T, 1.5) * lam / lam_ref;
  p11[5] = sqrt(T / q[5]);
  for (int k = 6; k < 11; ++k) p11[k] = q[k + 1];
}

bool quench_family(int family) { return family == FK_RUNAWAY_QUENCH_3D; }
bool runaway_family(int family) {
  return family == FK_RUNAWAY_3D || family == FK_RUNAWAY_QUENCH_3D;
}

// The static runaway constants of plan p at step n (t_n = n dt).
void runaway_params_at(const fk_plan* p, int n, double* p11) {
  if (quench_family(p->coeffs.family))
    quench_params(p->coeffs.p, n * p->dt, p11);
  else
    for (int k = 0; k < 11; ++k) p11[k] = p->coeffs.p[k];
}

// Largest sigma_m and |b_m| over the nodes for the constants q11 (sigma_p
// and b depend on (p, xi) and (p, r) only, so the pairs of axis nodes cover
// the mesh); running maxima in smax, bmax.
void runaway_bounds_at(const fk_plan* p, const double* q11, double* smax, double* bmax) {
  const int n0 = p->grid.n[0], n1 = p->grid.n[1], n2 = p->grid.n[2];
  auto x = [&](int m, int i) {
    return p->nu ? p->hcoord[m][i] : p->grid.lo[m] + (double)i * p->h[m];
  };
  double b[3], s[3];
  for (int i = 0; i < n0; ++i) {
    for (int j = 0; j < n1; ++j) {
      runaway_host(q11, x(0, i), x(1, j), x(2, 0), b, s);
      for (int m = 0; m < 2; ++m) {
        smax[m] = std::max(smax[m], s[m]);
        bmax[m] = std::max(bmax[m], fabs(b[m]));
      }
    }
    for (int k = 0; k < n2; ++k) {
      runaway_host(q11, x(0, i), 0.0, x(2, k), b, s);
      smax[2] = std::max(smax[2], s[2]);
      bmax[2] = std::max(bmax[2], fabs(b[2]));
    }
  }
}

// The same over every time step of a quench plan.
void runaway_bounds(const fk_plan* p, double* smax, double* bmax) {
  for (int m = 0; m < 3; ++m) smax[m] = bmax[m] = 0.0;
  const int times = quench_family(p->coeffs.family) ? p->n_steps : 1;
  for (int n = 0; n < times; ++n) {
    double q11[11];
    runaway_params_at(p, n, q11);
    runaway_bounds_at(p, q11, smax, bmax);
  }
}

fk_status validate(const fk_grid* g, const fk_region* r, const fk_coeffs* c, int q, double dt,
                   int n_steps, fk_precision prec, fk_path path) {
  if (!g || !c) return FK_ERR_INVALID_ARG;
  if (g->dim < 1 || g->dim > 3) return FK_ERR_INVALID_ARG;
  for (int m = 0; m < g->dim; ++m) {
    if (g->n[m] < 3) return FK_ERR_INVALID_ARG;
    if (!finite(g->lo[m]) || !finite(g->hi[m]) || !(g->hi[m] > g->lo[m])) return FK_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !finite(dt) || n_steps < 1) return FK_ERR_INVALID_ARG;
  if (prec != FK_FP32 && prec != FK_FP64) return FK_ERR_INVALID_ARG;
  if (path != FK_PATH_MATRIX_FREE && path != FK_PATH_CSR) return FK_ERR_INVALID_ARG;
  if (c->family != FK_CONST_DRIFT && c->family != FK_CELLULAR_FLOW &&
      c->family != FK_PAPER_CELLULAR && !runaway_family(c->family))
    return FK_ERR_INVALID_ARG;
  for (int k = 0; k < 16; ++k)
    if (!finite(c->p[k])) return FK_ERR_INVALID_ARG;
  if (c->family == FK_CONST_DRIFT && !(c->p[3] >= 0.0)) return FK_ERR_INVALID_ARG;
  if (c->family == FK_CELLULAR_FLOW && !(c->p[3] >= 0.0)) return FK_ERR_INVALID_ARG;
  if ((c->family == FK_CELLULAR_FLOW || c->family == FK_PAPER_CELLULAR) && g->dim != 2)
    return FK_ERR_INVALID_ARG;
  if (runaway_family(c->family)) {
    // x = (p, xi, r): p > 0, xi in [-1, 1], r >= 0; tau, W, Delta_p > 0,
    // the other rates non-negative (the quench variant: at t = 0; its
    // temperatures, t_star and mc2 positive)
    if (g->dim != 3) return FK_ERR_INVALID_ARG;
    if (!(g->lo[0] > 0.0) || !(g->lo[1] >= -1.0) || !(g->hi[1] <= 1.0) || !(g->lo[2] >= 0.0))
      return FK_ERR_INVALID_ARG;
    const double* q = c->p;
    if (quench_family(c->family)) {
      for (int k : {3, 4, 5, 6, 12})
        if (!(q[k] > 0.0)) return FK_ERR_INVALID_ARG;
      // ln Lambda must stay positive at every temperature the schedule
      // passes (T between T0 and Tf) and at Ttilde
      const double c0 = 14.9 - 0.5 * log(0.28);
      for (int k : {3, 4, 5})
        if (!(c0 + log(q[k]) > 0.0)) return FK_ERR_INVALID_ARG;
    }
    double q11[11];
    if (quench_family(c->family))
      quench_params(q, 0.0, q11);
    else
      for (int k = 0; k < 11; ++k) q11[k] = q[k];
    if (!(q11[1] > 0.0) || !(q11[7] > 0.0) || !(q11[8] > 0.0)) return FK_ERR_INVALID_ARG;
    if (!(q11[2] >= 0.0) || !(q11[3] >= 0.0) || !(q11[4] >= 0.0) || !(q11[5] >= 0.0) ||
        !(q11[10] >= 0.0))
      return FK_ERR_INVALID_ARG;
  }
  if (g->dim == 3) {
    // d = 3: constant drift or the runaway model on a uniform mesh,
    // matrix-free (the window kernel of fk_march3d.cuh)
    if ((c->family != FK_CONST_DRIFT && !runaway_family(c->family)) ||
        path != FK_PATH_MATRIX_FREE)
      return FK_ERR_UNSUPPORTED;
    if (r && r->absorbing_faces != FK_ALL_FACES_ABSORBING) return FK_ERR_UNSUPPORTED;
    for (int m = 0; m < 3; ++m)
      if (g->n[m] > 65535) return FK_ERR_UNSUPPORTED;
  }
  if (q < 1 || q > (g->dim == 1 ? FK_MAXQ : FK_MAXQ_2D)) return FK_ERR_UNSUPPORTED;
  if (r && r->absorbing_faces != FK_ALL_FACES_ABSORBING) {
    if (r->absorbing_faces != FK_PERIODIC_X || g->dim != 2 || path != FK_PATH_MATRIX_FREE)
      return FK_ERR_UNSUPPORTED;
  }
  bool nu = false;
  for (int m = 0; m < g->dim; ++m) {
    const double* ax = g->axis[m];
    if (!ax) continue;
    nu = true;
    if (ax[0] != g->lo[m] || ax[g->n[m] - 1] != g->hi[m]) return FK_ERR_INVALID_ARG;
    for (int i = 0; i + 1 < g->n[m]; ++i)
      if (!finite(ax[i + 1]) || !(ax[i + 1] > ax[i])) return FK_ERR_INVALID_ARG;
  }
  if (nu && (path != FK_PATH_MATRIX_FREE ||
             (r && r->absorbing_faces != FK_ALL_FACES_ABSORBING)))
    return FK_ERR_UNSUPPORTED;
  if (path == FK_PATH_CSR) {
    if (g->dim != 2 || c->family == FK_PAPER_CELLULAR) return FK_ERR_UNSUPPORTED;
    if (c->family == FK_CELLULAR_FLOW && c->p[1] != 0.0) return FK_ERR_UNSUPPORTED;
  }
  int64_t J = 1;
  for (int m = 0; m < g->dim; ++m) J *= g->n[m];
  if (J > ((int64_t)1 << 31) - 1) return FK_ERR_UNSUPPORTED;
  return FK_OK;
}

void free_coords(fk_plan* p) {
  for (int m = 0; m < 3; ++m) {
    free(p->hcoord[m]);
    p->hcoord[m] = nullptr;
  }
}

fk_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FK_OK;
  if (e == cudaErrorMemoryAllocation) return FK_ERR_OOM;
  return FK_ERR_CUDA;
}

// Node coordinates of a non-uniform plan, in the plan's precision (and, for
// an FP32 plan in d = 3, in FP64 as well: the runaway coefficients are
// evaluated at the FP64 node coordinates).
template <typename T>
fk_status upload_coords(fk_plan* p) {
  for (int m = 0; m < p->grid.dim; ++m) {
    const int nm = p->grid.n[m];
    std::vector<T> c(nm);
    for (int i = 0; i < nm; ++i) c[i] = (T)p->hcoord[m][i];
    fk_status st = fk_dev_alloc(p, &p->dcoord[m], sizeof(T) * nm);
    if (st == FK_OK)
      st = cuda_status(cudaMemcpy(p->dcoord[m], c.data(), sizeof(T) * nm, cudaMemcpyHostToDevice));
    if (st == FK_OK && p->grid.dim == 3 && sizeof(T) == 4) {
      st = fk_dev_alloc(p, &p->dcoord64[m], sizeof(double) * nm);
      if (st == FK_OK)
        st = cuda_status(cudaMemcpy(p->dcoord64[m], p->hcoord[m], sizeof(double) * nm,
                                    cudaMemcpyHostToDevice));
    }
    if (st != FK_OK) return st;
  }
  return FK_OK;
}

template <typename T>
fk_status upload_tables(fk_plan* p) {
  const int nx = p->grid.n[0], ny = p->grid.dim == 2 ? p->grid.n[1] : 1;
  T* ct = (T*)malloc(sizeof(T) * 4 * nx);
  T* rt = (T*)malloc(sizeof(T) * 2 * ny);
  if (!ct || !rt) {
    free(ct);
    free(rt);
    return FK_ERR_OOM;
  }
  // periodic x: column nx-1 is column 0 (its entries are node 0's)
  const int per = p->periodic_x ? nx - 1 : nx;
  const double nk = p->coeffs.p[1];
  for (int i = 0; i < nx; ++i) {
    const double x = p->nu ? p->hcoord[0][i] : p->grid.lo[0] + (i % per) * p->h[0];
    if (p->coeffs.family == FK_PAPER_CELLULAR) {
      // v_1 ~ sin(n x) + eps f cos(n x), v_2 ~ cos(n x) + eps f (-sin(n x))
      ct[4 * i + 0] = (T)sin(nk * x);
      ct[4 * i + 1] = (T)cos(nk * x);
      ct[4 * i + 2] = (T)cos(nk * x);
      ct[4 * i + 3] = (T)(-sin(nk * x));
    } else {
      ct[4 * i + 0] = (T)sin(kPi * x);
      ct[4 * i + 1] = (T)sin(2.0 * kPi * x);
      ct[4 * i + 2] = (T)cos(kPi * x);
      ct[4 * i + 3] = (T)cos(2.0 * kPi * x);
    }
  }
  for (int k = 0; k < ny; ++k) {
    const double y = p->grid.dim == 2 ? (p->nu ? p->hcoord[1][k] : p->grid.lo[1] + k * p->h[1])
                                      : 0.0;
    rt[2 * k + 0] = (T)cos(kPi * y);
    rt[2 * k + 1] = (T)sin(kPi * y);
  }
  fk_status st = fk_dev_alloc(p, &p->col_tab, sizeof(T) * 4 * nx);
  if (st == FK_OK) st = fk_dev_alloc(p, &p->row_tab, sizeof(T) * 2 * ny);
  if (st == FK_OK) st = cuda_status(cudaMemcpy(p->col_tab, ct, sizeof(T) * 4 * nx, cudaMemcpyHostToDevice));
  if (st == FK_OK) st = cuda_status(cudaMemcpy(p->row_tab, rt, sizeof(T) * 2 * ny, cudaMemcpyHostToDevice));
  free(ct);
  free(rt);
  return st;
}

template <typename T>
void fill2d(const fk_plan* p, int n, Step2D<T>* a) {
  memset(a, 0, sizeof(*a));
  a->ncols = 1;
  a->nx = p->grid.n[0];
  a->ny = p->grid.n[1];
  a->tx = p->tile[0];
  a->ty = p->tile[1];
  a->variant = p->variant;
  a->hx = p->halo[0];
  a->hy = p->halo[1];
  a->lx = a->tx + 2 * a->hx + 2;
  a->ly = a->ty + 2 * a->hy + 2;
  a->lyr = a->ly | 1;
  // drift form in the kernels: FK_CONST_DRIFT constants, else the
  // row x column tables (both cellular families)
  a->family = p->coeffs.family == FK_CONST_DRIFT ? FK_CONST_DRIFT : FK_CELLULAR_FLOW;
  a->px = p->periodic_x;
  const double dt = p->dt, tn = n * dt;
  // lengths in cells on a uniform mesh; physical lengths on a non-uniform one
  const double hx = p->nu ? 1.0 : p->h[0], hy = p->nu ? 1.0 : p->h[1];
  if (p->coeffs.family == FK_PAPER_CELLULAR) {
    // dx = Pe dt/h (-pi cos(pi y)) (sin(n x) + eps f cos(n x)),
    // dy = Pe dt/h (n sin(pi y)) (cos(n x) - eps f sin(n x)), f = cos(omega t)
    const double Pe = p->coeffs.p[0], nk = p->coeffs.p[1], eps = p->coeffs.p[2];
    const double f = cos(p->coeffs.p[3] * tn);
    a->kx = (T)(-Pe * kPi * dt / hx);
    a->ky = (T)(Pe * nk * dt / hy);
    a->A = (T)1.0;
    a->e1 = (T)(eps * f);
    a->e2 = (T)(eps * f);
  } else if (p->coeffs.family == FK_CELLULAR_FLOW) {
    const double A = p->coeffs.p[0], eps = p->coeffs.p[1], om = p->coeffs.p[2];
    const double st = sin(om * tn);
    a->kx = (T)(-kPi * dt / hx);
    a->ky = (T)(kPi * dt / hy);
    a->A = (T)A;
    a->e1 = (T)(eps * st);
    a->e2 = (T)(2.0 * eps * st);
  } else {
    a->cdx = (T)(p->coeffs.p[0] * dt / hx);
    a->cdy = (T)(p->coeffs.p[1] * dt / hy);
  }
  a->col_tab = (const T*)p->col_tab;
  a->row_tab = (const T*)p->row_tab;
  const double sg = sigma_of(&p->coeffs) * sqrt(2.0 * dt);
  for (int q = 0; q < p->q; ++q) {
    a->gx[q] = (T)(sg * p->gh_a[q] / hx);
    a->gy[q] = (T)(sg * p->gh_a[q] / hy);
    a->w[q] = (T)p->gh_w[q];
  }
  a->err = p->d_err;
  if (p->nu) {
    a->nu = 1;
    a->xc = (const T*)p->dcoord[0];
    a->yc = (const T*)p->dcoord[1];
    for (int m = 0; m < 2; ++m) {
      a->blo[m] = (T)p->grid.lo[m];
      a->bhi[m] = (T)p->grid.hi[m];
    }
  }
  a->win = (sizeof(T) == 4) ? p->win : 0;
  a->mode = a->win > 0 ? 1 : 0;
  if (a->win > 0) {
    a->row_lo = p->win_row_lo;
    a->row_hi = p->win_row_hi;
    a->nb_lo = (a->row_lo - 1 + a->ty - 1) / a->ty;
    for (int q = 0; q < p->q; ++q) a->wm[q] = p->wm[q];
  }
  if (p->use_masked && p->mwin > 0) {
    a->mode = 2;
    a->win = p->mwin;
    a->hx = p->mhalo[0];
    a->hy = p->mhalo[1];
    a->lx = fk_step2dm_lx(a->hx, a->win);
    a->ly = a->ty + 2 * a->hy + 2;
    a->lyr = a->lx;  // row pitch of the records
    a->mpat = p->mpat;
    for (int q = 0; q < p->q; ++q) {
      a->wm[q] = p->mwm[q];
      a->wmf[q] = (T)p->mwm[q];
      // g_q - m_q from the rounded offsets g_q (exact: m_q is an integer no
      // larger than the spread), so that the points stay symmetric
      a->gmx[q] = a->gx[q] - (T)p->mwm[q];
      a->gmy[q] = a->gy[q] - (T)p->mwm[q];
    }
  }
}

template <typename T>
void fill1d(const fk_plan* p, Step1D<T>* a) {
  memset(a, 0, sizeof(*a));
  a->ncols = 1;
  a->nx = p->grid.n[0];
  a->tx = p->tile[0];
  a->hx = p->halo[0];
  a->lx = a->tx + 2 * a->hx + 2;
  // lengths in cells on a uniform mesh; physical lengths on a non-uniform one
  const double hx = p->nu ? 1.0 : p->h[0];
  a->cdx = (T)(p->coeffs.p[0] * p->dt / hx);
  const double sg = sigma_of(&p->coeffs) * sqrt(2.0 * p->dt);
  for (int q = 0; q < p->q; ++q) {
    a->g[q] = (T)(sg * p->gh_a[q] / hx);
    a->w[q] = (T)p->gh_w[q];
  }
  a->err = p->d_err;
  if (p->nu) {
    a->nu = 1;
    a->xc = (const T*)p->dcoord[0];
    a->blo = (T)p->grid.lo[0];
    a->bhi = (T)p->grid.hi[0];
  }
}

// Candidate tiles of the 2D step kernel: 32 columns x ty rows, ty = 8 m,
// times the FP32 register-budget variants.  The first entry that fits is
// the default when no timing is done.
struct TileCand {
  int ty, variant;
};
const TileCand kCands[] = {{16, 0}, {8, 0}, {24, 0}, {32, 0}, {40, 0}, {48, 0}, {64, 0},
                           {16, 1}, {8, 1},  {24, 1}, {32, 1}, {48, 1}};

// Step kernels of a 2D plan: 0 direct, 1 row window (+ direct face bands),
// 2 masked tensor window.
enum { kDirect = 0, kRowWindow = 1, kMasked = 2 };

bool kernel_eligible(const fk_plan* p, int kern) {
  return kern == kDirect || (kern == kRowWindow && p->win_max > 0) ||
         (kern == kMasked && p->mwin > 0);
}

bool cand_fits(const fk_plan* p, const TileCand& c, int dev_smem, int kern = kDirect) {
  if (p->elem == 8 && c.variant != 0) return false;
  if (c.variant == 2 && kern != kMasked) return false;  // (4 CTAs/SM: masked FP32 only)
  // (two nodes per thread: masked FP32 with W = 7, even tile heights)
  if (c.variant == 3 && (kern != kMasked || p->mwin != 7 || c.ty % 2 != 0)) return false;
  if (kern == kMasked) {
    const int lx = fk_step2dm_lx(p->mhalo[0], p->mwin), ly = c.ty + 2 * p->mhalo[1] + 2;
    const size_t bytes = p->elem == 8 ? fk_step2dm64_smem(ly, lx) : fk_step2dm_smem(ly, lx);
    return bytes <= (size_t)dev_smem;
  }
  const int hy = p->halo[1] + (kern == kRowWindow ? 1 : 0);
  const int lx = 32 + 2 * p->halo[0] + 2, ly = c.ty + 2 * hy + 2;
  return fk_step2d_smem(lx, ly, ly | 1, p->elem, p->nu) <= (size_t)dev_smem;
}

void set_kernel(fk_plan* p, int kern) {
  p->win = kern == kRowWindow ? p->win_max : 0;
  p->use_masked = kern == kMasked ? 1 : 0;
}

int current_kernel(const fk_plan* p) {
  return p->use_masked ? kMasked : (p->win > 0 ? kRowWindow : kDirect);
}

// The window kernel (FP32, 2D, matrix-free) evaluates each cell row once per
// x-point.  It needs: a rule size it is built for; the y-cell offsets
// m_q = floor(gy_q - gy_0) of the points robustly integral-part-stable (the
// fractional part of gy_q - gy_0 away from 0 and 1, so that the actual cell
// offset of point q is m_q or m_q + 1 for every drift); fewer window rows
// W = m_{Q-1} + 3 than the direct form's 2Q row reads; and a non-empty band
// of rows whose points all stay strictly inside the box along y.
void window_eligibility(fk_plan* p) {
  p->win_max = 0;
  if (p->grid.dim != 2 || p->prec != FK_FP32 || p->path != FK_PATH_MATRIX_FREE) return;
  if (p->periodic_x || p->nu) return;  // periodic x, non-uniform: the direct kernel only
  const double sg = sigma_of(&p->coeffs) * sqrt(2.0 * p->dt);
  float gy[FK_MAXQ_2D];
  for (int q = 0; q < p->q; ++q) gy[q] = (float)(sg * p->gh_a[q] / p->h[1]);
  p->wm[0] = 0;  // point 0 defines the window origin
  for (int q = 1; q < p->q; ++q) {
    const double d = (double)gy[q] - (double)gy[0];
    const double f = d - floor(d);
    if (f < 1e-4 || f > 1.0 - 1e-4) return;
    p->wm[q] = (int)floor(d);
  }
  const int W = p->wm[p->q - 1] + 3;
  if (W >= 2 * p->q || !fk_window_available(p->q, W)) return;
  const int band = (int)ceil(p->reach[1] * (1.0 + 1e-6) + 1e-3) + 1;
  p->win_row_lo = band;
  p->win_row_hi = p->grid.n[1] - 1 - band;
  if (p->win_row_hi - p->win_row_lo < 8) return;
  p->win_max = W;
}

// The masked tensor-window kernels (FP32 and FP64, 2D, matrix-free) need: the cell
// offsets m_q = floor(g_q - g_0) the same on both axes (one uniform scatter
// pattern for the x and the y weights) with the fractional part of
// g_q - g_0 away from 0 and 1 by a margin that the FP32 rounding of the
// shifted positions cannot cross (then the cell of point q is m_q or
// m_q + 1 after the cell of point 0 for every drift); and a window width
// W = m_{Q-1} + 3 it is built for.  Its halo H = floor(reach) + 2 keeps
// the whole W x W window of every node of a tile inside the staged nodes.
void masked_eligibility(fk_plan* p) {
  const double kMargin = 1e-4;
  p->mwin = 0;
  if (p->grid.dim != 2 || p->path != FK_PATH_MATRIX_FREE) return;
  if (p->periodic_x || p->nu) return;  // periodic x, non-uniform: the direct kernel only
  const double sg = sigma_of(&p->coeffs) * sqrt(2.0 * p->dt);
  double gx[FK_MAXQ_2D], gy[FK_MAXQ_2D];  // the offsets as the kernel holds them
  for (int q = 0; q < p->q; ++q) {
    gx[q] = sg * p->gh_a[q] / p->h[0];
    gy[q] = sg * p->gh_a[q] / p->h[1];
    if (p->prec == FK_FP32) {
      gx[q] = (double)(float)gx[q];
      gy[q] = (double)(float)gy[q];
    }
  }
  p->mwm[0] = 0;
  for (int q = 1; q < p->q; ++q) {
    const double dx = gx[q] - gx[0], dy = gy[q] - gy[0];
    const double fx = dx - floor(dx), fy = dy - floor(dy);
    if (fx < kMargin || fx > 1.0 - kMargin || fy < kMargin || fy > 1.0 - kMargin) return;
    if (floor(dx) != floor(dy)) return;
    p->mwm[q] = (int)floor(dy);
  }
  const int W = p->mwm[p->q - 1] + 3;
  if (!fk_masked_available(p->q, W)) return;
  p->mpat = fk_masked_pattern(p->q, W, p->mwm);
  if (p->mpat < 0) return;
  for (int m = 0; m < 2; ++m) {
    // |error of a position difference| <= 2 ulp(reach + 1) << margin
    const double ulp2 = p->prec == FK_FP32 ? 4.8e-7 : 4.5e-16;
    if ((p->reach[m] + 1.0) * ulp2 > 0.5 * kMargin) return;
    const double r = p->reach[m] * (1.0 + 1e-6) + 1e-3;
    p->mhalo[m] = (int)floor(r) + 2;
  }
  if (32 + 2 * p->mhalo[0] + 2 > 2 + FK_THREADS) return;  // adjoint: one column per thread
  // step: the staging sweeps cover the pair columns with 31 per warp
  if (fk_step2dm_lx(p->mhalo[0], W) - 3 > 31 * (FK_THREADS / 32)) return;
  p->mwin = W;
}

// Choose the output tile and check the shared-memory budget.
fk_status choose_tiles(fk_plan* p) {
  int dev_smem = 0;
  cudaError_t e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  if (e != cudaSuccess) return FK_ERR_CUDA;
  if (p->grid.dim == 3) return FK_OK;  // no tiles: records are read through L1/L2
  if (p->grid.dim == 1) {
    // enough CTAs to spread a short line over the SMs (2 per SM), 32..1024 nodes each
    const int interior = p->grid.n[0] - 2;
    int t = (interior + 2 * 152 - 1) / (2 * 152);
    t = (t + 31) / 32 * 32;
    p->tile[0] = t < 32 ? 32 : (t > 1024 ? 1024 : t);
    const int lx = p->tile[0] + 2 * p->halo[0] + 2;
    if (fk_step1d_smem(lx, p->elem, p->nu) > (size_t)dev_smem) return FK_ERR_UNSUPPORTED;
    return FK_OK;
  }
  for (const TileCand& c : kCands) {
    if (cand_fits(p, c, dev_smem)) {
      p->tile[0] = 32;
      p->tile[1] = c.ty;
      p->variant = c.variant;
      return FK_OK;
    }
  }
  return FK_ERR_UNSUPPORTED;
}

// Autotuner: time one step of every fitting candidate (tile height x
// register budget x step kernel) on this device, from the terminal
// indicator, and keep the fastest.  Results are cached per problem shape
// for the life of the process.
struct TuneEntry {
  int dev, nx, ny, q, elem, hx, hy, family;
  int ty, variant, kern;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune_cache;

// The first fitting tile of the kernel in use (after an explicit kernel
// choice that the tuned tile does not fit).
void refit_tile(fk_plan* p) {
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  const int kern = current_kernel(p);
  if (cand_fits(p, TileCand{p->tile[1], p->variant}, dev_smem, kern)) return;
  for (const TileCand& c : kCands) {
    if (cand_fits(p, c, dev_smem, kern)) {
      p->tile[1] = c.ty;
      p->variant = c.variant;
      return;
    }
  }
  set_kernel(p, kDirect);
}

// Tile candidates of the masked kernel: the fixed list, three heights of
// variant 2 and four of variant 3, and tile heights that make the number of
// tiles just fit 1-4 waves of resident CTAs (3 per SM for variant 0, 2 for
// variants 1 and 3, 4 for variant 2), so that the last wave is not short
// (variant 3: rounded up to an even height).
std::vector<TileCand> masked_cands(const fk_plan* p) {
  std::vector<TileCand> v(std::begin(kCands), std::end(kCands));
  v.insert(v.end(), {TileCand{16, 2}, TileCand{24, 2}, TileCand{32, 2}, TileCand{16, 3},
                     TileCand{32, 3}, TileCand{48, 3}, TileCand{64, 3}});
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    sms = 152;
  const int nxt = (p->grid.n[0] - 2 + 31) / 32, rows = p->grid.n[1] - 2;
  for (int var = 0; var < 4; ++var) {
    const int per_sm = var == 0 ? 3 : var == 2 ? 4 : 2;
    for (int waves = 1; waves <= 4; ++waves) {
      const int row_tiles = waves * sms * per_sm / nxt;
      if (row_tiles < 1) continue;
      int ty = (rows + row_tiles - 1) / row_tiles;
      if (var == 3) ty += ty & 1;
      if (ty < 4 || ty > 64) continue;
      bool seen = false;
      for (const TileCand& c : v) seen = seen || (c.ty == ty && c.variant == var);
      if (!seen) v.push_back(TileCand{ty, var});
    }
  }
  return v;
}

// Mean time in ms of one replay of the work `enqueue` puts on stream s,
// captured once into a CUDA graph (a warm-up replay, then `reps` timed):
// fk_solve replays its march from a graph too, so host launch overhead,
// which on a fast step exceeds the step itself, stays out of the
// comparison.  1e30 when the capture, the instantiation or a replay fails
// (a configuration the device refuses); the error is cleared.
template <typename F>
float graph_ms(cudaStream_t s, int reps, F&& enqueue) {
  float ms = 1e30f;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return ms;
  }
  const fk_status es = enqueue();
  const cudaError_t ec = cudaStreamEndCapture(s, &g);
  if (es != FK_OK || ec != cudaSuccess || !g || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return ms;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess) {
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = cudaGraphLaunch(ge, s) == cudaSuccess;
    float t = 0.f;
    if (ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
      ms = t / reps;
  }
  cudaStreamSynchronize(s);
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  return ms;
}

fk_status autotune(fk_plan* p) {
  if (p->grid.dim != 2 || p->path != FK_PATH_MATRIX_FREE) return FK_OK;
  // explicit choice (profiling runs, where timing is distorted):
  // FK_STEP_TILE=ty[,variant[,kernel]], kernel 0 direct, 1 row window, 2 masked window
  if (const char* t = getenv("FK_STEP_TILE")) {
    int ty = 0, var = 0, kern = 0;
    if (sscanf(t, "%d,%d,%d", &ty, &var, &kern) >= 1 && ty >= 4 && ty <= 64 &&
        (var >= 0 && var <= 3) && kern >= 0 && kern <= 2) {
      if (kern != kMasked && ty % 8 != 0) ty = (ty + 7) / 8 * 8;
      int dev_smem = 0;
      cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
      const TileCand c = {ty, p->elem == 8 ? 0 : var};
      if (!kernel_eligible(p, kern)) kern = kDirect;
      if (cand_fits(p, c, dev_smem, kern)) {
        p->tile[1] = c.ty;
        p->variant = c.variant;
        set_kernel(p, kern);
        return FK_OK;
      }
    }
  }
  // small meshes are launch-bound: keep the default tile, prefer the masked kernel
  if (p->J_int < 16384) {
    if (p->mwin > 0) {
      set_kernel(p, kMasked);
      refit_tile(p);
    }
    return FK_OK;
  }
  TuneEntry key = {p->device, p->grid.n[0], p->grid.n[1], p->q, p->elem, p->halo[0], p->halo[1],
                   p->coeffs.family, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneEntry& t : g_tune_cache) {
      if (t.dev == key.dev && t.nx == key.nx && t.ny == key.ny && t.q == key.q &&
          t.elem == key.elem && t.hx == key.hx && t.hy == key.hy && t.family == key.family) {
        p->tile[1] = t.ty;
        p->variant = t.variant;
        set_kernel(p, kernel_eligible(p, t.kern) ? t.kern : kDirect);
        return FK_OK;
      }
    }
  }
  int dev_smem = 0;
  if (cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) !=
      cudaSuccess)
    return FK_ERR_CUDA;
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, (size_t)(p->J * p->elem)) != cudaSuccess) {
    cudaGetLastError();
    return FK_OK;  // keep the default tile
  }
  cudaStream_t s = p->cap_stream;
  fk_status st = cuda_status(
      fk_launch_fill_chi(p->scratch, 2, p->grid.n[0], p->grid.n[1], p->elem, s, p->periodic_x));
  if (st == FK_OK) st = cuda_status(cudaStreamSynchronize(s));
  const bool log = getenv("FK_TUNE_LOG") != nullptr;
  if (log)
    fprintf(stderr,
            "fk autotune %dx%d q=%d: row window %d (0: not eligible), band [%d, %d); "
            "masked window %d, halo %d %d\n",
            p->grid.n[0], p->grid.n[1], p->q, p->win_max, p->win_row_lo, p->win_row_hi, p->mwin,
            p->mhalo[0], p->mhalo[1]);
  float best = 1e30f;
  int best_ty = p->tile[1], best_var = p->variant, best_kern = kDirect;
  for (int kern = kDirect; kern <= kMasked; ++kern) {
    if (!kernel_eligible(p, kern)) continue;
    const std::vector<TileCand> cands =
        kern == kMasked ? masked_cands(p) : std::vector<TileCand>(std::begin(kCands), std::end(kCands));
    for (const TileCand& c : cands) {
      if (st != FK_OK) break;
      if (!cand_fits(p, c, dev_smem, kern)) continue;
      p->tile[1] = c.ty;
      p->variant = c.variant;
      set_kernel(p, kern);
      // 8 steps from chi per replay, 3 replays
      const int steps = 8;
      const float ms = graph_ms(s, 3, [&]() {
        fk_status e = FK_OK;
        for (int r = 0; r < steps && e == FK_OK; ++r)
          e = fk_enqueue_step(p, p->n_steps - 1, p->scratch, tmp, nullptr, s);
        return e;
      }) / steps;
      if (log)
        fprintf(stderr, "fk autotune %dx%d q=%d elem=%d: ty=%d variant=%d kernel=%d  %.2f us\n",
                p->grid.n[0], p->grid.n[1], p->q, p->elem, c.ty, c.variant, kern, ms * 1e3f);
      if (ms < best) {
        best = ms;
        best_ty = c.ty;
        best_var = c.variant;
        best_kern = kern;
      }
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  p->tile[1] = best_ty;
  p->variant = best_var;
  set_kernel(p, best_kern);
  cudaMemset(p->d_err, 0, sizeof(unsigned));
  if (st == FK_OK) {
    key.ty = best_ty;
    key.variant = best_var;
    key.kern = best_kern;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back(key);
  }
  return st;
}

fk_status enqueue_march(fk_plan* p, int n_from, int n_to, const void* u_in, void* u_out,
                        void* snaps, int stride, cudaStream_t s);
bool use_persistent(const fk_plan* p, const void* snaps, int steps);

// The persistent march's workspace: one flag per tile of the shortest tile
// candidate (4 rows) and the abort word, and the per-step drift factors
// (the same values the per-step launches receive).
fk_status persist_workspace(fk_plan* p) {
  p->mflags_n = (int64_t)((p->grid.n[0] - 2 + 31) / 32) * ((p->grid.n[1] - 2 + 3) / 4) + 1;
  fk_status st = fk_dev_alloc(p, (void**)&p->mflags, sizeof(unsigned) * p->mflags_n);
  if (st == FK_OK) st = fk_dev_alloc(p, (void**)&p->me12, sizeof(float2) * p->n_steps);
  if (st != FK_OK) return st;
  std::vector<float2> e(p->n_steps);
  for (int n = 0; n < p->n_steps; ++n) {
    Step2D<float> a;
    fill2d<float>(p, n, &a);
    e[n] = make_float2(a.e1, a.e2);
  }
  return cuda_status(
      cudaMemcpy(p->me12, e.data(), sizeof(float2) * p->n_steps, cudaMemcpyHostToDevice));
}

// Whole marches of a masked-kernel plan: the persistent march or one
// launch per step, whichever a short timed march (min(N, 16) steps from
// chi) finds faster.  FK_MARCH=persistent|steps chooses explicitly.
fk_status tune_persist(fk_plan* p) {
  p->persist = 0;
  if (!p->mflags || !p->use_masked || p->mwin <= 0) return FK_OK;
  const char* f = getenv("FK_MARCH");
  if (f && strcmp(f, "steps") == 0) return FK_OK;
  const int steps = p->n_steps < 16 ? p->n_steps : 16;
  p->persist = 1;
  if (!use_persistent(p, nullptr, steps)) {
    p->persist = 0;
    return FK_OK;
  }
  if (f && strcmp(f, "persistent") == 0) return FK_OK;
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, (size_t)(p->J * p->elem)) != cudaSuccess) {
    cudaGetLastError();
    p->persist = 0;
    return FK_OK;
  }
  cudaStream_t s = p->cap_stream;
  float ms[2] = {1e30f, 1e30f};
  fk_status st = FK_OK;
  const bool log = getenv("FK_TUNE_LOG") != nullptr;
  // each mode as fk_solve replays it: a graph of the march from chi (a
  // persistent launch that the device refuses times as 1e30: the per-step
  // launches stay)
  for (int mode = 0; mode < 2; ++mode) {
    p->persist = mode;
    ms[mode] = graph_ms(s, 2, [&]() {
      fk_status e = cuda_status(
          fk_launch_fill_chi(p->scratch, 2, p->grid.n[0], p->grid.n[1], p->elem, s));
      if (e == FK_OK)
        e = enqueue_march(p, p->n_steps, p->n_steps - steps, p->scratch, tmp, nullptr, 0, s);
      return e;
    });
  }
  if (log)
    fprintf(stderr, "fk march tune %dx%d: %d steps, per-step launches %.1f us, persistent %.1f us\n",
            p->grid.n[0], p->grid.n[1], steps, ms[0] * 1e3f, ms[1] * 1e3f);
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  cudaMemset(p->d_err, 0, sizeof(unsigned));
  p->persist = (st == FK_OK && ms[1] < ms[0]) ? 1 : 0;
  return st;
}

}  // namespace

// ------------------------------------------------------------ internal --

namespace {
std::mutex g_alloc_mu;
long g_alloc_fail_at = 0, g_alloc_count = 0;  // FK_TEST_FAIL_ALLOC state
}  // namespace

fk_status fk_dev_alloc(fk_plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return FK_OK;
  {
    const char* f = getenv("FK_TEST_FAIL_ALLOC");
    const long n = f ? atol(f) : 0;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (n != g_alloc_fail_at) {  // set, changed or cleared: count afresh
      g_alloc_fail_at = n;
      g_alloc_count = 0;
    }
    if (n > 0 && ++g_alloc_count == n) return FK_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FK_ERR_OOM : FK_ERR_CUDA;
  }
  p->workspace_bytes += (int64_t)bytes;
  return FK_OK;
}

void fk_dev_free(void* ptr) {
  if (ptr) cudaFree(ptr);
}

void fk_fill_step2d_f32(const fk_plan* p, int n, Step2D<float>* a) { fill2d<float>(p, n, a); }
void fk_fill_step2d_f64(const fk_plan* p, int n, Step2D<double>* a) { fill2d<double>(p, n, a); }

namespace {
template <typename T>
void fill3d(const fk_plan* p, int n, Step3D<T>* a) {
  memset(a, 0, sizeof(*a));
  a->rec = (V4<T>*)p->rec3d;
  a->nx = p->grid.n[0];
  a->ny = p->grid.n[1];
  a->nz = p->grid.n[2];
  a->q = p->q;
  a->w3 = p->w3;
  const double sg = sigma_of(&p->coeffs) * sqrt(2.0 * p->dt);
  for (int m = 0; m < 3; ++m) {
    // in cells of a uniform mesh, physical lengths on a non-uniform one
    const double hm = p->nu ? 1.0 : p->h[m];
    a->cd[m] = (T)(p->coeffs.p[m] * p->dt / hm);
    a->gs[m] = (T)(sg / hm);
  }
  if (p->nu) {
    a->nu = 1;
    for (int m = 0; m < 3; ++m) {
      a->xc[m] = (const T*)p->dcoord[m];
      a->xd[m] = (const double*)(sizeof(T) == 8 ? p->dcoord[m] : p->dcoord64[m]);
    }
  }
  for (int q = 0; q < p->q; ++q) {
    a->ga[q] = (T)p->gh_a[q];
    a->gw[q] = (T)p->gh_w[q];
  }
  a->err = p->d_err;
  // both runaway variants run the runaway kernel; the quench variant with
  // the constants of t_n = n dt
  const bool re = runaway_family(p->coeffs.family);
  a->family = re ? FK_RUNAWAY_3D : p->coeffs.family;
  for (int m = 0; m < 3; ++m) {
    a->lo[m] = p->grid.lo[m];
    a->h[m] = p->h[m];
    // faces: every one exits with 1, except in the runaway model (p_max 1,
    // p_min and the wall 0, xi and r = r_lo reflect)
    a->face[m][0] = !re ? FK_FACE_EXIT1 : (m == 0 ? FK_FACE_EXIT0 : FK_FACE_REFLECT);
    a->face[m][1] = !re ? FK_FACE_EXIT1
                        : (m == 0 ? FK_FACE_EXIT1 : (m == 1 ? FK_FACE_REFLECT : FK_FACE_EXIT0));
    a->first[m] = a->face[m][0] == FK_FACE_REFLECT ? 0 : 1;
    const int last = a->face[m][1] == FK_FACE_REFLECT ? p->grid.n[m] - 1 : p->grid.n[m] - 2;
    a->count[m] = last - a->first[m] + 1;
  }
  if (re) runaway_params_at(p, n, a->rp);
  a->dt = (T)p->dt;
  a->sq2dt = (T)sqrt(2.0 * p->dt);
  a->coef = (const T*)p->coef3d;
  a->coef_per_step = quench_family(p->coeffs.family) ? 1 : 0;
}

// The runaway model's per-node coefficients (Eq. (ex32d)), six values per
// node that the step reads: the static model's once per plan here, the
// quench variant's by each step at its t_n.
template <typename T>
fk_status fill_coef3d(fk_plan* p) {
  fk_status st = fk_dev_alloc(p, &p->coef3d, (size_t)(6 * p->J * p->elem));
  if (st != FK_OK || quench_family(p->coeffs.family)) return st;
  Step3D<T> a;
  fill3d<T>(p, 0, &a);
  st = cuda_status(fk_launch_coef3d<T>(a, (T*)p->coef3d, 0));
  if (st == FK_OK) st = cuda_status(cudaDeviceSynchronize());
  return st;
}

// The terminal indicator of a 3D plan into u (device, J values).
fk_status chi3d(const fk_plan* p, void* u, cudaStream_t s) {
  cudaError_t e;
  if (p->prec == FK_FP32) {
    Step3D<float> a;
    fill3d<float>(p, 0, &a);
    e = fk_launch_chi3d<float>(a, (float*)u, s);
  } else {
    Step3D<double> a;
    fill3d<double>(p, 0, &a);
    e = fk_launch_chi3d<double>(a, (double*)u, s);
  }
  return cuda_status(e);
}

// One step of each of nfields fields (J values apart): the record pass and
// the window pass per field (the records are one field's workspace).
template <typename T>
cudaError_t step3d(const fk_plan* p, int n, const void* u_in, void* u_out, void* snap, int nfields,
                   cudaStream_t s) {
  Step3D<T> a;
  fill3d<T>(p, n, &a);
  for (int f = 0; f < nfields; ++f) {
    a.u_in = (const T*)u_in + (int64_t)f * p->J;
    a.u_out = (T*)u_out + (int64_t)f * p->J;
    a.snap = (T*)snap;
    cudaError_t e = fk_launch_step3d<T>(a, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

fk_status enqueue_step(fk_plan* p, int n, const void* u_in, void* u_out, void* snap,
                       int nfields, cudaStream_t s) {
  cudaError_t e;
  if (p->grid.dim == 3) {
    e = p->prec == FK_FP32 ? step3d<float>(p, n, u_in, u_out, snap, nfields, s)
                           : step3d<double>(p, n, u_in, u_out, snap, nfields, s);
    return cuda_status(e);
  }
  if (p->grid.dim == 2) {
    if (p->prec == FK_FP32) {
      Step2D<float> a;
      fill2d<float>(p, n, &a);
      a.u_in = (const float*)u_in;
      a.u_out = (float*)u_out;
      a.snap = (float*)snap;
      a.ncols = nfields;
      a.zstride = nfields > 1 ? p->J : 0;
      e = fk_launch_step2d<float>(a, p->q, s);
    } else {
      Step2D<double> a;
      fill2d<double>(p, n, &a);
      a.u_in = (const double*)u_in;
      a.u_out = (double*)u_out;
      a.snap = (double*)snap;
      a.ncols = nfields;
      a.zstride = nfields > 1 ? p->J : 0;
      e = fk_launch_step2d<double>(a, p->q, s);
    }
  } else {
    if (p->prec == FK_FP32) {
      Step1D<float> a;
      fill1d<float>(p, &a);
      a.u_in = (const float*)u_in;
      a.u_out = (float*)u_out;
      a.snap = (float*)snap;
      a.ncols = nfields;
      a.zstride = nfields > 1 ? p->J : 0;
      e = fk_launch_step1d<float>(a, p->q, s);
    } else {
      Step1D<double> a;
      fill1d<double>(p, &a);
      a.u_in = (const double*)u_in;
      a.u_out = (double*)u_out;
      a.snap = (double*)snap;
      a.ncols = nfields;
      a.zstride = nfields > 1 ? p->J : 0;
      e = fk_launch_step1d<double>(a, p->q, s);
    }
  }
  return cuda_status(e);
}
}  // namespace

fk_status fk_enqueue_step(fk_plan* p, int n, const void* u_in, void* u_out, void* snap,
                          cudaStream_t s) {
  if (p->path == FK_PATH_CSR) return fk_csr_step(p, u_in, u_out, snap, s);
  return enqueue_step(p, n, u_in, u_out, snap, 1, s);
}

fk_status fk_enqueue_step_fields(fk_plan* p, int n, const void* u_in, void* u_out, int nfields,
                                 cudaStream_t s) {
  if (p->path == FK_PATH_CSR || nfields < 1) return FK_ERR_UNSUPPORTED;
  return enqueue_step(p, n, u_in, u_out, nullptr, nfields, s);
}

namespace {

// Steps n_from-1 .. n_to from u_in (NULL = chi) into u_out, ping-ponging
// between u_out and the plan's scratch field so that the last step lands in
// u_out; snapshots as documented for fk_solve when snaps != NULL.
// Whether a march of `steps` steps runs as the masked kernel's persistent
// march: an FP32 2D plan on the masked kernel that chose it, no snapshots,
// not inside a batch, tiles taller than their halo, and every tile
// resident at once.
bool use_persistent(const fk_plan* p, const void* snaps, int steps) {
  if (!p->persist || p->no_persist || snaps || steps < 2 || !p->use_masked || p->mwin <= 0 ||
      p->prec != FK_FP32 || p->grid.dim != 2 || !p->mflags || !p->me12)
    return false;
  Step2D<float> a;
  fill2d<float>(p, 0, &a);
  // a tile waits for the 3 x 3 block of tiles around it only: its staged
  // halo must stay within that block
  if (a.hy + 1 > a.ty || a.hx + 1 > 32) return false;
  const int64_t tiles = (int64_t)((a.nx - 2 + 31) / 32) * ((a.ny - 2 + a.ty - 1) / a.ty);
  return tiles + 1 <= p->mflags_n && fk_march2dm_fits(a, p->q);
}

fk_status enqueue_march(fk_plan* p, int n_from, int n_to, const void* u_in, void* u_out,
                        void* snaps, int stride, cudaStream_t s) {
  const int64_t bytes = p->J * p->elem;
  const int steps = n_from - n_to;
  if (steps == 0) {
    if (!u_in) {
      if (p->grid.dim == 3) return chi3d(p, u_out, s);
      return cuda_status(fk_launch_fill_chi(u_out, p->grid.dim, p->grid.n[0], p->grid.n[1],
                                            p->elem, s, p->periodic_x));
    }
    if (u_in != u_out) return cuda_status(fk_launch_copy(u_out, u_in, bytes, s));
    return FK_OK;
  }
  if (p->grid.dim == 1 && p->resident1d) {
    cudaError_t e;
    const int c = p->resident1d == 2 ? p->cluster1d : 0;
    if (p->prec == FK_FP32) {
      Step1D<float> a;
      fill1d<float>(p, &a);
      e = c ? fk_launch_march1d_cluster<float>(a, p->q, c, (const float*)u_in, (float*)u_out,
                                               (float*)snaps, stride, steps, s)
            : fk_launch_march1d<float>(a, p->q, (const float*)u_in, (float*)u_out,
                                       (float*)snaps, stride, steps, s);
    } else {
      Step1D<double> a;
      fill1d<double>(p, &a);
      e = c ? fk_launch_march1d_cluster<double>(a, p->q, c, (const double*)u_in, (double*)u_out,
                                                (double*)snaps, stride, steps, s)
            : fk_launch_march1d<double>(a, p->q, (const double*)u_in, (double*)u_out,
                                        (double*)snaps, stride, steps, s);
    }
    return cuda_status(e);
  }
  const bool first_to_out = ((steps - 1) % 2) == 0;  // does step 1 write u_out?
  const void* src = u_in;
  if (!src) {
    void* buf = first_to_out ? p->scratch : u_out;
    fk_status st = p->grid.dim == 3
                       ? chi3d(p, buf, s)
                       : cuda_status(fk_launch_fill_chi(buf, p->grid.dim, p->grid.n[0],
                                                        p->grid.n[1], p->elem, s, p->periodic_x));
    if (st != FK_OK) return st;
    src = buf;
  } else if (src == u_out && first_to_out) {
    fk_status st = cuda_status(fk_launch_copy(p->scratch, src, bytes, s));
    if (st != FK_OK) return st;
    src = p->scratch;
  }
  if (use_persistent(p, snaps, steps)) {
    // the whole march in one launch (fk_window.cuh): tile flags and the
    // abort word start at zero
    Step2D<float> a;
    fill2d<float>(p, n_from - 1, &a);
    MaskedMarch mm;
    mm.u_first = (const float*)src;
    mm.buf[0] = (float*)u_out;
    mm.buf[1] = (float*)p->scratch;
    mm.e12 = p->me12;
    mm.flags = p->mflags;
    mm.abort = p->mflags + p->mflags_n - 1;
    mm.n_from = n_from;
    mm.steps = steps;
    // test hook: tile 0 never publishes a step, so the tiles around it run
    // into their wait limit (the timeout path)
    mm.silent = getenv("FK_TEST_STALL_MARCH") ? 0 : -1;
    cudaError_t e = cudaMemsetAsync(p->mflags, 0, sizeof(unsigned) * p->mflags_n, s);
    if (e == cudaSuccess) e = fk_launch_march2dm(a, mm, p->q, s);
    return cuda_status(e);
  }
  for (int m = 1; m <= steps; ++m) {
    const int n = n_from - m;
    void* dst = ((steps - m) % 2 == 0) ? u_out : p->scratch;
    void* snap = nullptr;
    if (snaps && stride > 0 && (m % stride) == 0)
      snap = (char*)snaps + (int64_t)(m / stride - 1) * bytes;
    fk_status st = fk_enqueue_step(p, n, src, dst, snap, s);
    if (st != FK_OK) return st;
    src = dst;
  }
  return FK_OK;
}

}  // namespace

// ------------------------------------------------------------- the ABI --

extern "C" {

const char* fk_status_string(fk_status s) {
  switch (s) {
    case FK_OK: return "FK_OK";
    case FK_ERR_INVALID_ARG: return "FK_ERR_INVALID_ARG: invalid argument";
    case FK_ERR_UNSUPPORTED: return "FK_ERR_UNSUPPORTED: case not implemented";
    case FK_ERR_OOM: return "FK_ERR_OOM: device allocation failed";
    case FK_ERR_CUDA: return "FK_ERR_CUDA: CUDA runtime error";
    case FK_ERR_TIMEOUT: return "FK_ERR_TIMEOUT: bounded device wait expired";
    case FK_ERR_DEVICE: return "FK_ERR_DEVICE: device-side range check fired";
  }
  return "unknown fk_status";
}

fk_status fk_gauss_hermite(int q, double* a, double* w) {
  if (!a || !w || q < 1 || q > FK_MAXQ) return FK_ERR_INVALID_ARG;
  return gauss_hermite(q, a, w) ? FK_OK : FK_ERR_INVALID_ARG;
}

fk_status fk_runaway_quench_params(const double* p13, double t, double* p11) {
  auto fin = [](double v) { return v == v && v - v == 0.0; };
  if (!p13 || !p11 || !fin(t)) return FK_ERR_INVALID_ARG;
  for (int k : {3, 4, 5, 6, 12})
    if (!(p13[k] > 0.0) || !fin(p13[k])) return FK_ERR_INVALID_ARG;
  quench_params(p13, t, p11);
  return FK_OK;
}

fk_status fk_plan_create(fk_plan** out, const fk_grid* grid, const fk_region* region,
                         const fk_coeffs* coeffs, int q_per_dim, double dt, int n_steps,
                         fk_precision prec, fk_path path) {
  FkRange range("fk_plan_create");
  if (!out) return FK_ERR_INVALID_ARG;
  *out = nullptr;
  fk_status st = validate(grid, region, coeffs, q_per_dim, dt, n_steps, prec, path);
  if (st != FK_OK) return st;
  fk_plan* p = new (std::nothrow) fk_plan;
  if (!p) return FK_ERR_OOM;
  memset(p, 0, sizeof(*p));
  p->grid = *grid;
  for (int m = grid->dim; m < 3; ++m) {
    p->grid.n[m] = 1;
    p->grid.lo[m] = 0.0;
    p->grid.hi[m] = 0.0;
  }
  // non-uniform axes: the plan keeps its own copy of every axis (the
  // uniform ones written out) and drops the caller's pointers
  for (int m = 0; m < 3; ++m) p->grid.axis[m] = nullptr;
  for (int m = 0; m < grid->dim; ++m) p->nu |= grid->axis[m] ? 1 : 0;
  if (p->nu) {
    for (int m = 0; m < grid->dim; ++m) {
      const int nm = grid->n[m];
      p->hcoord[m] = (double*)malloc(sizeof(double) * nm);
      if (!p->hcoord[m]) {
        free_coords(p);
        delete p;
        return FK_ERR_OOM;
      }
      for (int i = 0; i < nm; ++i)
        p->hcoord[m][i] = grid->axis[m] ? grid->axis[m][i]
                                        : grid->lo[m] + i * (grid->hi[m] - grid->lo[m]) / (nm - 1);
    }
  }
  p->region.absorbing_faces = region ? region->absorbing_faces : FK_ALL_FACES_ABSORBING;
  p->periodic_x = p->region.absorbing_faces == FK_PERIODIC_X ? 1 : 0;
  p->coeffs = *coeffs;
  p->q = q_per_dim;
  p->dt = dt;
  p->n_steps = n_steps;
  p->prec = prec;
  p->path = path;
  p->elem = prec == FK_FP32 ? 4 : 8;
  if (!gauss_hermite(q_per_dim, p->gh_a, p->gh_w)) {
    free_coords(p);
    delete p;
    return FK_ERR_INVALID_ARG;
  }
  p->J = 1;
  p->J_int = 1;
  for (int m = 0; m < grid->dim; ++m) {
    p->J *= grid->n[m];
    p->J_int *= grid->n[m] - 2;
    p->h[m] = (grid->hi[m] - grid->lo[m]) / (grid->n[m] - 1);
  }
  // halo: every shifted point of an interior node stays within
  // [i - halo + 1, i + halo - 1] cells, so its cell and the cell's right
  // node are staged, and so are their slope stencils.
  double bmax[3];
  drift_bound(coeffs, grid->dim, bmax);
  const double amax = fabs(p->gh_a[0]);
  const double sg = sigma_of(coeffs) * sqrt(2.0 * dt);
  for (int m = 0; m < grid->dim; ++m) {
    p->reach[m] = (bmax[m] * dt + sg * amax) / p->h[m];
    const double r = p->reach[m] * (1.0 + 1e-6) + 1e-3;
    if (r > 4096.0) {
      free_coords(p);
      delete p;
      return FK_ERR_UNSUPPORTED;
    }
    p->halo[m] = (int)ceil(r) + 1;
    if (p->nu) {
      // every shifted point of node i lies within R of x_i: its cell c must
      // satisfy i - halo <= c <= i + halo - 1 (the cells staged around i)
      const double* x = p->hcoord[m];
      const int nm = grid->n[m];
      const double R = (bmax[m] * dt + sg * amax) * (1.0 + 1e-6) + 1e-12;
      auto cell = [&](double z) {
        int lo = 0, up = nm - 1;
        while (up - lo > 1) {
          const int mid = (lo + up) / 2;
          if (x[mid] <= z) lo = mid; else up = mid;
        }
        return lo;  // in [0, nm-2]
      };
      int h = 1;
      for (int i = 0; i < nm; ++i) {
        const int cl = cell(x[i] - R), cr = cell(x[i] + R);
        h = std::max(h, std::max(i - cl, cr + 1 - i));
      }
      p->halo[m] = h + 1;  // one more for FP32 rounding of the positions
      p->reach[m] = h;
      if (p->halo[m] > 4096) {
        free_coords(p);
        delete p;
        return FK_ERR_UNSUPPORTED;
      }
    }
  }
  // periodic x: a staged column wraps by at most one period
  if (p->periodic_x && p->halo[0] + 2 >= grid->n[0] - 1) {
    free_coords(p);
    delete p;
    return FK_ERR_UNSUPPORTED;
  }
  if (grid->dim == 3) {
    // window width: the points of one axis span gs (a_{Q-1} - a_0) cells
    // and touch at most floor(span) + 2 cells, W = floor(span) + 3 nodes
    // (a small margin covers rounding of the positions).  The runaway
    // model takes the largest span over the nodes, and its mirrored points
    // reach |shift| + span / 2 cells into the box from a reflecting face.
    int w = 3;
    double smax[3], bmax3[3];
    if (runaway_family(coeffs->family)) {
      runaway_bounds(p, smax, bmax3);
    } else {
      for (int m = 0; m < 3; ++m) {
        smax[m] = sigma_of(coeffs);
        bmax3[m] = fabs(coeffs->p[m]);
      }
    }
    for (int m = 0; m < 3; ++m) {
      if (p->nu) {
        // non-uniform axis: every point of node i (mirrored ones included)
        // lies within R of x_i and in the box, so its window covers the
        // cells of [max(lo, x_i - R), min(hi, x_i + R)] and their right
        // nodes
        const double* x = p->hcoord[m];
        const int nm = grid->n[m];
        const double L = x[nm - 1] - x[0];
        const double R = (bmax3[m] * dt + 0.5 * smax[m] * sqrt(2.0 * dt) *
                                              (p->gh_a[q_per_dim - 1] - p->gh_a[0])) *
                             (1.0 + 1e-6) + 1e-6 * L;
        auto cell = [&](double z) {
          int lo = 0, up = nm - 1;
          while (up - lo > 1) {
            const int mid = (lo + up) / 2;
            if (x[mid] <= z) lo = mid; else up = mid;
          }
          return lo;  // in [0, nm-2]
        };
        int cells = 1;
        for (int i = 0; i < nm; ++i)
          cells = std::max(cells, cell(std::min(x[nm - 1], x[i] + R)) -
                                      cell(std::max(x[0], x[i] - R)) + 1);
        w = std::max(w, cells + 1);
        p->reach[m] = 0.5 * cells;
        p->halo[m] = cells + 1;
        continue;
      }
      const double span = smax[m] * sqrt(2.0 * dt) * (p->gh_a[q_per_dim - 1] - p->gh_a[0]) /
                          p->h[m];
      const double shift = bmax3[m] * dt / p->h[m];
      w = std::max(w, (int)floor(span * (1.0 + 1e-6) + 1e-3) + 3);
      if (runaway_family(coeffs->family))
        w = std::max(w, (int)floor((shift + 0.5 * span) * (1.0 + 1e-6) + 1e-3) + 2);
      p->reach[m] = shift + 0.5 * span;
      p->halo[m] = (int)ceil(p->reach[m]) + 1;
    }
    bool fits = w <= FK_MAXW_3D;
    for (int m = 0; m < 3; ++m) fits = fits && grid->n[m] >= w;
    if (!fits) {
      free_coords(p);
      delete p;
      return FK_ERR_UNSUPPORTED;
    }
    p->w3 = w;
  }
  window_eligibility(p);
  masked_eligibility(p);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    free_coords(p);
    delete p;
    return FK_ERR_CUDA;
  }
  st = choose_tiles(p);
  // the CSR path launches no step kernel: a halo too wide for any tile only
  // concerns the matrix-free path
  if (st == FK_ERR_UNSUPPORTED && path == FK_PATH_CSR) st = FK_OK;
  if (st == FK_OK && path == FK_PATH_MATRIX_FREE && grid->dim != 3)
    st = cuda_status(fk_prepare_step_kernels(grid->dim, q_per_dim, p->elem));
  if (st == FK_OK && grid->dim == 1) {
    // The whole 1D march in one launch: FP32 in one CTA when the field, its
    // second buffer and the slopes fit its shared memory; FP64 over a
    // cluster of up to 16 CTAs (at GB300's FP64 rate one SM is slower than
    // one launch per step spread over several SMs), about 16 nodes per CTA.
    // FK_1D_KERNEL=step|resident|cluster chooses explicitly (tests).
    const char* k = getenv("FK_1D_KERNEL");
    const int nx = grid->n[0];
    int want = prec == FK_FP32 ? 1 : 2;
    if (k && strcmp(k, "step") == 0) want = 0;
    if (k && strcmp(k, "resident") == 0) want = 1;
    if (k && strcmp(k, "cluster") == 0) want = 2;
    if (p->nu) want = 0;  // non-uniform: the per-step kernel only
    if (want == 1 && fk_march1d_smem(nx, p->elem) <= 200 * 1024) {
      st = cuda_status(fk_prepare_march1d(q_per_dim, p->elem));
      if (st == FK_OK) p->resident1d = 1;
    } else if (want == 2) {
      const int maxc = fk_prepare_march1d_cluster(q_per_dim, p->elem);
      int c = (nx + 15) / 16;
      if (c > maxc) c = maxc;
      const int chunk = c > 0 ? (nx + c - 1) / c : 0, L = chunk + 2 * (p->halo[0] + 2);
      if (c >= 1 && (size_t)(3 * L + chunk * q_per_dim) * p->elem <= 200 * 1024) {
        p->resident1d = 2;
        p->cluster1d = c;
      }
    }
  }
  if (st == FK_OK) st = fk_dev_alloc(p, (void**)&p->d_err, sizeof(unsigned));
  if (st == FK_OK) st = cuda_status(cudaMemset(p->d_err, 0, sizeof(unsigned)));
  if (st == FK_OK) st = fk_dev_alloc(p, &p->scratch, (size_t)(p->J * p->elem));
  if (st == FK_OK && grid->dim == 3)
    st = fk_dev_alloc(p, &p->rec3d, (size_t)(4 * p->J * p->elem));
  if (st == FK_OK) st = (prec == FK_FP32) ? upload_tables<float>(p) : upload_tables<double>(p);
  if (st == FK_OK && p->nu)
    st = (prec == FK_FP32) ? upload_coords<float>(p) : upload_coords<double>(p);
  if (st == FK_OK && grid->dim == 3 && runaway_family(p->coeffs.family))
    st = (prec == FK_FP32) ? fill_coef3d<float>(p) : fill_coef3d<double>(p);
  if (st == FK_OK) st = cuda_status(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  if (st == FK_OK && p->mwin > 0 && prec == FK_FP32 && grid->dim == 2) st = persist_workspace(p);
  if (st == FK_OK) st = autotune(p);
  if (st == FK_OK) st = tune_persist(p);
  if (st == FK_OK) {
    // explicit choice of the 2D step kernel (tests exercise both paths)
    const char* k = getenv("FK_STEP_KERNEL");
    int kern = -1;
    if (k && strcmp(k, "direct") == 0) kern = kDirect;
    if (k && strcmp(k, "window") == 0) kern = kRowWindow;
    if (k && strcmp(k, "masked") == 0) kern = kMasked;
    if (kern >= 0 && kernel_eligible(p, kern) && p->grid.dim == 2) {
      set_kernel(p, kern);
      refit_tile(p);
    }
  }
  if (st == FK_OK && path == FK_PATH_CSR) {
    st = fk_csr_assemble(p, p->cap_stream);
    if (st == FK_OK) st = cuda_status(cudaStreamSynchronize(p->cap_stream));
    unsigned h = 0;
    if (st == FK_OK) st = cuda_status(cudaMemcpy(&h, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st == FK_OK && h) st = FK_ERR_DEVICE;
  }
  if (st != FK_OK) {
    fk_plan_destroy(p);
    return st;
  }
  *out = p;
  return FK_OK;
}

fk_status fk_plan_destroy(fk_plan* p) {
  if (!p) return FK_OK;
  cudaDeviceSynchronize();
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  fk_dev_free(p->scratch);
  fk_dev_free(p->rec3d);
  fk_dev_free(p->coef3d);
  fk_dev_free(p->col_tab);
  fk_dev_free(p->row_tab);
  fk_dev_free(p->d_err);
  fk_dev_free(p->csr_rowptr);
  fk_dev_free(p->csr_val);
  fk_dev_free(p->csr_c);
  fk_dev_free(p->stack);
  fk_dev_free(p->batch_rec);
  fk_dev_free(p->hz_ws);
  fk_dev_free(p->host_io);
  for (int m = 0; m < 3; ++m) {
    fk_dev_free(p->dcoord[m]);
    fk_dev_free(p->dcoord64[m]);
  }
  free_coords(p);
  fk_dev_free(p->adj_ws);
  fk_dev_free(p->adj_tab);
  fk_dev_free(p->mflags);
  fk_dev_free(p->me12);
  for (int i = 0; i < p->adj_ev_cap; ++i) cudaEventDestroy(p->adj_ev[i]);
  free(p->adj_ev);
  for (int i = 0; i < p->adj_sev_n; ++i) cudaEventDestroy(p->adj_sev[i]);
  if (p->adj_s2) cudaStreamDestroy(p->adj_s2);
  fk_batch_release(p);
  delete p;
  return FK_OK;
}

fk_status fk_plan_get_info(const fk_plan* p, fk_plan_info* info) {
  if (!p || !info) return FK_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->n_nodes = p->J;
  info->n_interior = p->J_int;
  info->dim = p->grid.dim;
  info->q_per_dim = p->q;
  info->n_steps = p->n_steps;
  info->precision = p->prec;
  info->path = p->path;
  for (int m = 0; m < 3; ++m) {
    info->halo[m] = p->halo[m];
    info->tile[m] = p->tile[m];
    info->reach_cells[m] = p->reach[m];
  }
  info->csr_nnz = p->csr_nnz;
  info->workspace_bytes = p->workspace_bytes;
  info->window_rows = p->grid.dim == 3 ? p->w3 : (p->use_masked ? p->mwin : p->win);
  info->periodic_x = p->periodic_x;
  info->nonuniform = p->nu;
  info->step_kernel = p->grid.dim == 1   ? (p->resident1d ? 2 + p->resident1d : 0)
                      : p->grid.dim == 3 ? 5
                                         : current_kernel(p);
  info->batch_mode = fk_batch_mode(p);
  info->adjoint_kernel = p->adj_kernel;
  info->march_mode = p->persist ? 1 : 0;
  info->nodes_per_thread =
      p->grid.dim == 2 && p->use_masked && p->elem == 4 && p->variant == 3 ? 2 : 1;
  return FK_OK;
}

fk_status fk_march(fk_plan* p, int n_from, int n_to, const void* u_in, void* u_out,
                   cudaStream_t stream) {
  FkRange range("fk_march");
  if (!p || !u_in || !u_out) return FK_ERR_INVALID_ARG;
  if (n_to < 0 || n_from < n_to || n_from > p->n_steps) return FK_ERR_INVALID_ARG;
  return enqueue_march(p, n_from, n_to, u_in, u_out, nullptr, 0, stream);
}

fk_status fk_solve(fk_plan* p, const void* u_terminal, void* u_out, void* snapshots,
                   int snapshot_stride, cudaStream_t stream) {
  FkRange range("fk_solve");
  if (!p || !u_out) return FK_ERR_INVALID_ARG;
  if (snapshots && snapshot_stride < 1) return FK_ERR_INVALID_ARG;
  if (!snapshots) snapshot_stride = 0;
  const int pers = p->persist && !p->no_persist;
  const bool hit = p->graph && p->g_in == u_terminal && p->g_out == u_out &&
                   p->g_snap == snapshots && p->g_stride == snapshot_stride &&
                   p->g_persist == pers;
  if (!hit) {
    if (p->graph) {
      cudaGraphExecDestroy(p->graph);
      p->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return FK_ERR_CUDA;
    fk_status st = enqueue_march(p, p->n_steps, 0, u_terminal, u_out, snapshots,
                                 snapshot_stride, p->cap_stream);
    e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st != FK_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return FK_ERR_CUDA;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e);
    p->graph = ex;
    p->g_in = u_terminal;
    p->g_out = u_out;
    p->g_snap = snapshots;
    p->g_stride = snapshot_stride;
    p->g_persist = pers;
  }
  return cuda_status(cudaGraphLaunch(p->graph, stream));
}

fk_status fk_solve_host(fk_plan* p, const void* u_terminal_host, void* u_out_host,
                        cudaStream_t stream) {
  FkRange range("fk_solve_host");
  if (!p || !u_out_host) return FK_ERR_INVALID_ARG;
  const size_t bytes = (size_t)(p->J * p->elem);
  if (!p->host_io) {
    fk_status st = fk_dev_alloc(p, &p->host_io, bytes);
    if (st != FK_OK) return st;
  }
  if (u_terminal_host &&
      cudaMemcpyAsync(p->host_io, u_terminal_host, bytes, cudaMemcpyHostToDevice, stream) !=
          cudaSuccess)
    return FK_ERR_CUDA;
  // (in place on the device: fk_solve's march reads u^N before it writes u_out)
  fk_status st =
      fk_solve(p, u_terminal_host ? p->host_io : nullptr, p->host_io, nullptr, 0, stream);
  if (st != FK_OK) return st;
  if (cudaMemcpyAsync(u_out_host, p->host_io, bytes, cudaMemcpyDeviceToHost, stream) !=
      cudaSuccess)
    return FK_ERR_CUDA;
  return FK_OK;
}

// Algorithm 1 (Sec. 3.2).  Field c (1-based) starts in buffer c mod 2 (odd:
// the plan's second buffer, even: p_out) and takes one step at each loop
// index n = c, c-1, ..., 1, so at index n every active field has taken
// c - n steps and sits in buffer (c + c - n) mod 2 = n mod 2: all active
// fields read the same buffer and write the other, and after index 1 every
// field is in p_out.  Index n applies the step with the coefficients of
// t_{n-1}.
fk_status fk_solve_horizons(fk_plan* p, const void* u_terminal, void* p_out,
                            cudaStream_t stream) {
  FkRange range("fk_solve_horizons");
  if (!p || !p_out) return FK_ERR_INVALID_ARG;
  if (p->path != FK_PATH_MATRIX_FREE) return FK_ERR_UNSUPPORTED;
  const int N = p->n_steps;
  const int64_t fb = p->J * p->elem;
  const char* t0 = (const char*)u_terminal;
  const char* o0 = (const char*)p_out;
  if (t0 && t0 + fb > o0 && t0 < o0 + (int64_t)N * fb) return FK_ERR_INVALID_ARG;
  if (p->hz_bytes < (int64_t)N * fb) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FK_ERR_CUDA;
    fk_dev_free(p->hz_ws);
    p->hz_ws = nullptr;
    p->hz_bytes = 0;
    fk_status st = fk_dev_alloc(p, &p->hz_ws, (size_t)N * fb);
    if (st != FK_OK) return st;
    p->hz_bytes = (int64_t)N * fb;
  }
  char* buf[2] = {(char*)p_out, (char*)p->hz_ws};
  fk_status st = FK_OK;
  if (p->grid.dim == 3 && !u_terminal) {
    // the 3D indicator depends on the faces' exit values: form it once
    st = chi3d(p, p->scratch, stream);
    u_terminal = p->scratch;
  }
  if (st == FK_OK)
    st = cuda_status(fk_launch_fill_fields(buf[0], buf[1], u_terminal, p->grid.dim,
                                           p->grid.n[0], p->grid.n[1], p->elem, N, stream,
                                           p->periodic_x, p->grid.n[2]));
  const int kMaxFields = 65535;  // grid z limit
  for (int n = N; n >= 1 && st == FK_OK; --n) {
    const int par = n & 1;
    for (int c0 = n; c0 <= N && st == FK_OK; c0 += kMaxFields) {
      const int nf = N - c0 + 1 < kMaxFields ? N - c0 + 1 : kMaxFields;
      const int64_t off = (int64_t)(c0 - 1) * fb;
      st = fk_enqueue_step_fields(p, n - 1, buf[par] + off, buf[par ^ 1] + off, nf, stream);
    }
  }
  return st;
}

fk_status fk_last_device_error(fk_plan* p) {
  if (!p) return FK_ERR_INVALID_ARG;
  unsigned h = 0;
  cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return FK_ERR_CUDA;
  if (h) cudaMemset(p->d_err, 0, sizeof(unsigned));
  if (h & FK_DEVERR_TIMEOUT) return FK_ERR_TIMEOUT;
  if (h & FK_DEVERR_RANGE) return FK_ERR_DEVICE;
  return FK_OK;
}

}  // extern "C"
