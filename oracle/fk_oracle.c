/*
 * FP64 CPU oracle for the Feynman-Kac exit-probability march
 * (Yang, Zhang, del-Castillo-Negrete, Stoyanov, arXiv 2104.14561).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code with the CUDA path and is written to be checked against the paper
 * by eye: every query point is evaluated on its own, in the order Scheme 1
 * states, with no blocking, fusion or factorisation.
 *
 * What it computes (Sec. 3.1, Scheme 1), for n = n_from-1 down to n_to:
 *   Step 4 of the previous step / the terminal field: nodal slopes of u^{n+1}
 *          by the PCHIP rule Eq. (e300), one grid line at a time, with the
 *          end rule stated right after Eq. (e300);
 *   Step 1: z_{jq} = x_j + b(t_n,x_j) dt + sigma(t_n,x_j) sqrt(2 dt) a_q,
 *          Eq. (e31), over the tensor Gauss-Hermite rule of Eq. (quad);
 *   Step 2: the PCHIP interpolant of Eq. (Lag11) at z_{jq}; its 1D cell
 *          formula is the cubic Hermite formula of Sec. 3.1.2 and its
 *          multi-dimensional form the tensor product of that formula with
 *          nodal values and first partials only (the columns of Psi in
 *          Eq. (e34)); a query outside the closed box takes the exit value 1
 *          (Eq. (e24): the exit event contributes probability 1);
 *   Step 3: u^n_j = sum_q w_q u^{n+1,J}(z_{jq}), Eq. (e304);
 *   boundary nodes take u^n = 1 (Eq. (e3), Dirichlet value 1 on the boundary).
 *
 * An axis may instead be periodic (the x_1 direction of the paper's own 2D
 * example, Sec. 4.2): its two end nodes are the same point, the period is
 * the n - 1 distinct nodes, slopes and shifted points wrap around, and no
 * point exits through that axis.
 *
 * The runaway-electron model of Sec. 4.3 counts only exits through
 * p = p_max (value 1).  Its other faces follow the face rules of
 * face_rule() below: an exit through p = p_min or r = 1 takes the value 0,
 * and the faces xi = +-1 and r = 0, which the process does not cross,
 * mirror a shifted point back into the box.
 *
 * Readings where the paper is silent or garbled are documented next to the
 * code that takes them.  Coefficient time is the left end t_n = n dt
 * (Eq. (ref-X)).  Every floating-point value is IEEE binary64; the library
 * is built with -ffp-contract=off so that the host compiler does not fuse
 * multiply-adds behind the reader's back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FKO_MAXDIM 3
#define FKO_CONST_DRIFT 0
#define FKO_CELLULAR_FLOW 1
#define FKO_PAPER_CELLULAR 2
#define FKO_RUNAWAY 3
#define FKO_RUNAWAY_QUENCH 4

static const double FKO_PI = 3.14159265358979323846264338327950288;

typedef struct fko_grid {
  int dim;
  int n[FKO_MAXDIM];
  double lo[FKO_MAXDIM];
  double hi[FKO_MAXDIM];
  int periodic; /* bit m: axis m is periodic (node n-1 is node 0) */
  /* axis[m]: NULL for the uniform mesh, else the n[m] increasing node
   * coordinates of axis m (axis[m][0] = lo[m], axis[m][n-1] = hi[m]) */
  const double *axis[FKO_MAXDIM];
} fko_grid;

static int axis_periodic(const fko_grid *g, int m) { return (g->periodic >> m) & 1; }

/* ---------------------------------------------------------------- grid -- */

static int64_t grid_size(const fko_grid *g) {
  int64_t J = 1;
  for (int m = 0; m < g->dim; ++m) J *= g->n[m];
  return J;
}

static double grid_h(const fko_grid *g, int m) {
  return (g->hi[m] - g->lo[m]) / (double)(g->n[m] - 1);
}

/* Mesh S of Sec. 3.1.2: per axis either uniform, x_i = lo + i h, or the
 * given increasing coordinates (the partition along each direction need
 * not be uniform). */
static double grid_x(const fko_grid *g, int m, int i) {
  if (g->axis[m]) return g->axis[m][i];
  return g->lo[m] + (double)i * grid_h(g, m);
}

static int64_t grid_stride(const fko_grid *g, int m) {
  int64_t s = 1;
  for (int k = 0; k < m; ++k) s *= g->n[k];
  return s;
}

/* Multi-index of the scalar node number j (x fastest). */
static void grid_unflatten(const fko_grid *g, int64_t j, int *idx) {
  for (int m = 0; m < g->dim; ++m) {
    idx[m] = (int)(j % g->n[m]);
    j /= g->n[m];
  }
}

/* The node an update is computed at: the last node of a periodic axis is
 * node 0 (the same point), so it takes node 0's value. */
static void grid_canonical(const fko_grid *g, int *idx) {
  for (int m = 0; m < g->dim; ++m)
    if (axis_periodic(g, m) && idx[m] == g->n[m] - 1) idx[m] = 0;
}

/* What a face does to the process.  Every face of a non-periodic axis is
 * absorbing with exit value 1 (Eq. (e24)), except in the runaway-electron
 * model of Sec. 4.3, where only p = p_max (the upper face of axis 0) counts
 * as runaway: p = p_min and the wall r = 1 absorb with value 0, and the
 * faces xi = -1, xi = 1 and r = 0, which the process does not cross (the xi
 * diffusion vanishes there and the drift points inwards; r = 0 is the
 * axis), reflect. */
enum { FACE_EXIT0 = 0, FACE_EXIT1 = 1, FACE_REFLECT = 2 };
static int face_rule(int family, int m, int upper) {
  if (family != FKO_RUNAWAY && family != FKO_RUNAWAY_QUENCH) return FACE_EXIT1;
  if (m == 0) return upper ? FACE_EXIT1 : FACE_EXIT0;
  if (m == 1) return FACE_REFLECT;
  return upper ? FACE_EXIT0 : FACE_REFLECT;
}

/* Nodes on an absorbing face are boundary nodes; they hold the face's exit
 * value, 1 when any of their faces has value 1.  Returns -1 for a node the
 * scheme updates. */
static double boundary_value(const fko_grid *g, int family, const int *idx) {
  int on = 0, one = 0;
  for (int m = 0; m < g->dim; ++m) {
    if (axis_periodic(g, m)) continue;
    for (int up = 0; up < 2; ++up) {
      if (idx[m] != (up ? g->n[m] - 1 : 0)) continue;
      int rule = face_rule(family, m, up);
      if (rule == FACE_REFLECT) continue;
      on = 1;
      if (rule == FACE_EXIT1) one = 1;
    }
  }
  if (!on) return -1.0;
  return one ? 1.0 : 0.0;
}

static int grid_check(const fko_grid *g) {
  if (g->dim < 1 || g->dim > FKO_MAXDIM) return 1;
  for (int m = 0; m < g->dim; ++m) {
    if (g->n[m] < 3) return 1;
    if (!(g->hi[m] > g->lo[m])) return 1;
  }
  if (g->periodic & ~((1 << g->dim) - 1)) return 1;
  for (int m = 0; m < g->dim; ++m) {
    if (!g->axis[m]) continue;
    if (axis_periodic(g, m)) return 1; /* periodic axes are uniform */
    if (g->axis[m][0] != g->lo[m] || g->axis[m][g->n[m] - 1] != g->hi[m]) return 1;
    for (int i = 0; i + 1 < g->n[m]; ++i)
      if (!(g->axis[m][i + 1] > g->axis[m][i])) return 1;
  }
  if (g->periodic == (1 << g->dim) - 1) return 1; /* some face must absorb */
  return 0;
}

/* -------------------------------------------------------- coefficients -- */

/*
 * FKO_RUNAWAY_QUENCH (d = 3): the time-dependent runaway model at the end
 * of Sec. 4.3, p = (E_0, tau, Z, T0, Tf, Ttilde, t_star, r_D, W, Delta_p,
 * V_0, D_0, mc2).  The plasma temperature falls as
 *   T(t) = Tf + (T0 - Tf) exp(-t / t_star),
 * and with ln Lambda(T) = 14.9 - (1/2) ln 0.28 + ln T the constants of the
 * static model become
 *   v_T = sqrt(T / Ttilde),  nu_ee = (Ttilde / T)^{3/2} ln Lambda(T) / ln Lambda(Ttilde),
 *   delta = sqrt(2 T / mc2),  E = E_0 (T0 / T)^{3/2};
 * the remaining ones are taken as given.  Temperatures and mc2 share one
 * unit (keV: mc2 = 511).
 */
static void quench_static_params(const double *q, double t, double *p11) {
  const double T = q[4] + (q[3] - q[4]) * exp(-t / q[6]);
  const double lnL = 14.9 - 0.5 * log(0.28) + log(T);
  const double lnLt = 14.9 - 0.5 * log(0.28) + log(q[5]);
  p11[0] = q[0] * pow(q[3] / T, 1.5);          /* E */
  p11[1] = q[1];                               /* tau */
  p11[2] = q[2];                               /* Z */
  p11[3] = sqrt(2.0 * T / q[12]);              /* delta */
  p11[4] = pow(q[5] / T, 1.5) * lnL / lnLt;    /* nu_ee */
  p11[5] = sqrt(T / q[5]);                     /* v_T */
  p11[6] = q[7];                               /* r_D */
  p11[7] = q[8];                               /* W */
  p11[8] = q[9];                               /* Delta_p */
  p11[9] = q[10];                              /* V_0 */
  p11[10] = q[11];                             /* D_0 */
}

void fko_quench_params(const double *q, double t, double *p11) { quench_static_params(q, t, p11); }

/*
 * FKO_RUNAWAY (d = 3), x = (p, xi, r) (momentum, cosine of the pitch angle,
 * minor radius), parameters
 *   p = (E, tau, Z, delta, nu_ee, v_T, r_D, W, Delta_p, V_0, D_0):
 * Eq. (ex32d) of Sec. 4.3 with the collision functions
 *   C_A = nu v_T^2 psi(y) / y,
 *   C_B = (1/2) nu v_T^2 (1/y) [Z + phi(y) - psi(y) + y^2 delta^4 / 2],
 *   C_F = 2 nu v_T psi(y),
 *   phi = erf, psi(y) = [phi(y) - y phi'(y)] / (2 y^2),
 *   y = p / gamma, gamma = sqrt(1 + (delta p)^2),
 * and V(r) = V_0 1{r > r_D}, D(r, p) = (D_0/2)(1 + tanh((r - r_D)/W))
 * exp(-(p/Delta_p)^2).  The drift of p carries the derivative
 * (1/p^2) d/dp (p^2 C_A), written out by the chain rule:
 *   d/dp [p^2 psi(y) / y] = 2 p psi / y + p^2 (psi'/y - psi/y^2) dy/dp,
 *   dy/dp = 1/gamma^3,  psi'(y) = phi'(y) - 2 psi(y) / y.
 * sigma is diagonal: sqrt(2 C_A), sqrt(2 C_B) sqrt(1 - xi^2) / p,
 * sqrt(2 D).  The coefficients do not depend on t.
 */
static void runaway_coefficients(const double *p, const double *x, double *b, double *sig) {
  const double E = p[0], tau = p[1], Z = p[2], delta = p[3], nu = p[4], vT = p[5];
  const double rD = p[6], Wr = p[7], Dp = p[8], V0 = p[9], D0 = p[10];
  const double mom = x[0], xi = x[1], r = x[2];
  const double gam = sqrt(1.0 + (delta * mom) * (delta * mom));
  const double y = mom / gam;
  const double phi = erf(y);
  const double dphi = 2.0 / sqrt(FKO_PI) * exp(-y * y);
  const double psi = (phi - y * dphi) / (2.0 * y * y);
  const double dpsi = dphi - 2.0 * psi / y;
  const double CA = nu * vT * vT * psi / y;
  const double CB = 0.5 * nu * vT * vT / y * (Z + phi - psi + 0.5 * y * y * pow(delta, 4.0));
  const double CF = 2.0 * nu * vT * psi;
  const double dy = 1.0 / (gam * gam * gam);
  const double df = 2.0 * mom * psi / y + mom * mom * (dpsi / y - psi / (y * y)) * dy;
  const double dp2CA = nu * vT * vT * df; /* d/dp (p^2 C_A) */
  const double one_m = 1.0 - xi * xi;
  b[0] = E * xi - gam * mom / tau * one_m - CF + dp2CA / (mom * mom);
  b[1] = E * one_m / mom - xi * one_m / (tau * gam) - 2.0 * xi * CB / (mom * mom);
  const double th = tanh((r - rD) / Wr);
  const double ep = exp(-(mom / Dp) * (mom / Dp));
  const double D = 0.5 * D0 * (1.0 + th) * ep;
  const double dD = 0.5 * D0 * (1.0 - th * th) / Wr * ep;
  b[2] = (r > rD ? V0 : 0.0) + dD;
  sig[0] = sqrt(2.0 * CA);
  sig[4] = sqrt(2.0 * CB) * sqrt(one_m) / mom;
  sig[8] = sqrt(2.0 * D);
}

/*
 * Drift b(t,x) and diffusion matrix sigma(t,x) (d x d, row-major) of the
 * SDE Eq. (e1).
 *
 * FKO_CONST_DRIFT, p = (b_1, ..., b_d, s) with p[3] = s: b constant,
 *   sigma = s I.  (Sec. 4.1 is the case d = 1, b = 0, s = 1.)
 * FKO_CELLULAR_FLOW (d = 2), p = (A, eps, omega, D): the passive tracer of
 *   Sec. 4.2 in the stream-function form
 *     psi = A sin(pi x) sin(pi y) + eps sin(omega t) sin(2 pi x) sin(pi y),
 *   velocity b = (-d psi/dy, d psi/dx) (the orientation of the paper's
 *   cellular-flow velocity), and sigma = sqrt(2 D) I, so that the generator
 *   is b.grad + D Laplacian.
 * FKO_PAPER_CELLULAR (d = 2), p = (Pe, n, eps, omega): the paper's own
 *   example of Sec. 4.2, dx = Pe v dt + dW with
 *     v_1 = -pi cos(pi x_2) [sin(n x_1) + eps f(t) cos(n x_1)],
 *     v_2 =  n sin(pi x_2) [cos(n x_1) - eps f(t) sin(n x_1)],
 *   f(t) = cos(omega t), and sigma = I (unit Brownian motions).
 */
void fko_coefficients(int family, const double *p, int dim, double t,
                      const double *x, double *b, double *sig) {
  for (int i = 0; i < dim * dim; ++i) sig[i] = 0.0;
  if (family == FKO_CONST_DRIFT) {
    for (int m = 0; m < dim; ++m) {
      b[m] = p[m];
      sig[m * dim + m] = p[3];
    }
    return;
  }
  if (family == FKO_RUNAWAY) {
    runaway_coefficients(p, x, b, sig);
    return;
  }
  if (family == FKO_RUNAWAY_QUENCH) {
    double p11[11];
    quench_static_params(p, t, p11);
    runaway_coefficients(p11, x, b, sig);
    return;
  }
  if (family == FKO_PAPER_CELLULAR) {
    double Pe = p[0], nn = p[1], eps = p[2], omega = p[3];
    double f = cos(omega * t);
    double X = x[0], Y = x[1];
    b[0] = Pe * (-FKO_PI * cos(FKO_PI * Y) * (sin(nn * X) + eps * f * cos(nn * X)));
    b[1] = Pe * (nn * sin(FKO_PI * Y) * (cos(nn * X) - eps * f * sin(nn * X)));
    sig[0] = 1.0;
    sig[3] = 1.0;
    return;
  }
  /* FKO_CELLULAR_FLOW */
  {
    double A = p[0], eps = p[1], omega = p[2], D = p[3];
    double f = sin(omega * t);
    double X = x[0], Y = x[1];
    double dpsi_dy = FKO_PI * cos(FKO_PI * Y) *
                     (A * sin(FKO_PI * X) + eps * f * sin(2.0 * FKO_PI * X));
    double dpsi_dx = sin(FKO_PI * Y) * (A * FKO_PI * cos(FKO_PI * X) +
                                        eps * f * 2.0 * FKO_PI * cos(2.0 * FKO_PI * X));
    b[0] = -dpsi_dy;
    b[1] = dpsi_dx;
    sig[0] = sqrt(2.0 * D);
    sig[3] = sqrt(2.0 * D);
  }
}

static int family_check(int family, int dim, const double *p) {
  if (family == FKO_CONST_DRIFT) return !(p[3] >= 0.0);
  if (family == FKO_CELLULAR_FLOW) return dim != 2 || !(p[3] >= 0.0);
  if (family == FKO_PAPER_CELLULAR) return dim != 2;
  if (family == FKO_RUNAWAY || family == FKO_RUNAWAY_QUENCH) return dim != 3;
  return 1;
}

/* ---------------------------------------------------------- PCHIP (F) -- */

/*
 * Eq. (e300): the nodal derivative is 0 when the two neighbouring divided
 * differences have opposite signs, else their harmonic mean
 * 2 / (1/delta_{j-1} + 1/delta_j).  The paper does not say what happens when
 * one of them is zero; we read "opposite signs" as delta_{j-1} delta_j <= 0,
 * which is also the limit of the harmonic mean as either difference tends
 * to zero.
 */
static double pchip_rule(double d_left, double d_right) {
  if (d_left * d_right <= 0.0) return 0.0;
  return 2.0 / (1.0 / d_left + 1.0 / d_right);
}

/*
 * Nodal slopes of u along axis m for every node.  Interior nodes use
 * (delta_{i-1}, delta_i); the first node uses (delta_1, delta_2) and the
 * last node (delta_{J-1}, delta_{J-2}) in the paper's 1-based numbering of
 * the divided differences, i.e. (delta_0, delta_1) and (delta_{n-2},
 * delta_{n-3}) in 0-based numbering.  On a periodic axis every node is
 * interior: its neighbours are taken modulo the period n - 1.
 */
static void slopes_axis(const fko_grid *g, int m, const double *u, double *du) {
  int64_t J = grid_size(g);
  int64_t st = grid_stride(g, m);
  int nm = g->n[m];
  int idx[FKO_MAXDIM];
  for (int64_t j = 0; j < J; ++j) {
    grid_unflatten(g, j, idx);
    int i = idx[m];
    int64_t base = j - (int64_t)i * st; /* node 0 of this grid line */
#define U_(k) u[base + (int64_t)(k) * st]
#define DELTA(k) ((U_((k) + 1) - U_(k)) / (grid_x(g, m, (k) + 1) - grid_x(g, m, (k))))
    double d;
    if (axis_periodic(g, m)) {
      int P = nm - 1, ic = i % P;
      int il = (ic + P - 1) % P, ir = (ic + 1) % P;
      double h = grid_h(g, m); /* periodic axes are uniform */
      d = pchip_rule((U_(ic) - U_(il)) / h, (U_(ir) - U_(ic)) / h);
    } else if (i == 0)
      d = pchip_rule(DELTA(0), DELTA(1));
    else if (i == nm - 1)
      d = pchip_rule(DELTA(nm - 2), DELTA(nm - 3));
    else
      d = pchip_rule(DELTA(i - 1), DELTA(i));
#undef DELTA
#undef U_
    du[j] = d;
  }
}

void fko_slopes(const fko_grid *g, const double *u, double *du) {
  int64_t J = grid_size(g);
  for (int m = 0; m < g->dim; ++m) slopes_axis(g, m, u, du + (int64_t)m * J);
}

/*
 * The 1D cubic Hermite cell formula of Sec. 3.1.2 on [x_c, x_c + h] with
 * s = z - x_c, written as the four basis functions that multiply
 * u_c, u_{c+1}, u'_c, u'_{c+1}.
 */
static void hermite_basis(double s, double h, double *phi0, double *phi1,
                          double *psi0, double *psi1) {
  double h3 = h * h * h, h2 = h * h;
  *phi1 = (3.0 * h * s * s - 2.0 * s * s * s) / h3;
  *phi0 = (h3 - 3.0 * h * s * s + 2.0 * s * s * s) / h3;
  *psi1 = s * s * (s - h) / h2;
  *psi0 = s * (s - h) * (s - h) / h2;
}

/*
 * u^{n,J}(z) of Eq. (Lag11) for z in the closed box: the tensor product of
 * the 1D Hermite formula, carrying the nodal value and the d first partials
 * at each of the 2^d corners of the cell that contains z.  The cell is
 * floor((z - lo)/h) clamped to [0, n-2]; the interpolant is C^1 across cell
 * faces, so a point on a face gets the same value from either side.
 */
static double interpolate(const fko_grid *g, const double *u, const double *du,
                          const double *z) {
  int64_t J = grid_size(g);
  int c[FKO_MAXDIM];
  double phi[FKO_MAXDIM][2], psi[FKO_MAXDIM][2];
  for (int m = 0; m < g->dim; ++m) {
    int cm;
    if (g->axis[m]) {
      /* the last node at or left of z (bisection), clamped to a cell */
      int a = 0, b = g->n[m] - 1;
      while (b - a > 1) {
        int mid = (a + b) / 2;
        if (g->axis[m][mid] <= z[m]) a = mid; else b = mid;
      }
      cm = a;
    } else {
      cm = (int)floor((z[m] - g->lo[m]) / grid_h(g, m));
    }
    if (cm < 0) cm = 0;
    if (cm > g->n[m] - 2) cm = g->n[m] - 2;
    c[m] = cm;
    double h = grid_x(g, m, cm + 1) - grid_x(g, m, cm);
    double s = z[m] - grid_x(g, m, cm);
    hermite_basis(s, h, &phi[m][0], &phi[m][1], &psi[m][0], &psi[m][1]);
  }
  double value = 0.0;
  for (int corner = 0; corner < (1 << g->dim); ++corner) {
    int64_t node = 0;
    for (int m = 0; m < g->dim; ++m) {
      int bit = (corner >> m) & 1;
      node += (int64_t)(c[m] + bit) * grid_stride(g, m);
    }
    /* value basis: product of phi over all axes */
    double wv = 1.0;
    for (int m = 0; m < g->dim; ++m) wv *= phi[m][(corner >> m) & 1];
    value += wv * u[node];
    /* derivative basis along axis m: psi on axis m, phi on the others */
    for (int m = 0; m < g->dim; ++m) {
      double wd = 1.0;
      for (int k = 0; k < g->dim; ++k) {
        int bit = (corner >> k) & 1;
        wd *= (k == m) ? psi[k][bit] : phi[k][bit];
      }
      value += wd * du[(int64_t)m * J + node];
    }
  }
  return value;
}

/* --------------------------------------------------------- one node ---- */

/*
 * Steps 1-3 of Scheme 1 for one node: the tensor Gauss-Hermite sum of the
 * interpolant at the shifted points, exit value 1 outside the closed box.
 * a[], w[] hold the 1D rule normalised to the density pi^{-1/2} exp(-xi^2)
 * (Eq. (expec)), so the tensor weights are products of w and sum to 1.
 */
static double node_update(const fko_grid *g, int family, const double *p,
                          int nq, const double *a, const double *w, double dt,
                          double tn, const double *u, const double *du,
                          const int *idx) {
  int d = g->dim;
  double x[FKO_MAXDIM], b[FKO_MAXDIM], sig[FKO_MAXDIM * FKO_MAXDIM];
  for (int m = 0; m < d; ++m) x[m] = grid_x(g, m, idx[m]);
  fko_coefficients(family, p, d, tn, x, b, sig);
  double sq = sqrt(2.0 * dt);
  int64_t nqd = 1;
  for (int m = 0; m < d; ++m) nqd *= nq;
  double sum = 0.0;
  for (int64_t qq = 0; qq < nqd; ++qq) {
    int q[FKO_MAXDIM];
    int64_t r = qq;
    double wq = 1.0;
    for (int m = 0; m < d; ++m) {
      q[m] = (int)(r % nq);
      r /= nq;
      wq *= w[q[m]];
    }
    double z[FKO_MAXDIM];
    int outside = 0, exit_one = 0;
    for (int m = 0; m < d; ++m) {
      double noise = 0.0;
      for (int k = 0; k < d; ++k) noise += sig[m * d + k] * a[q[k]];
      z[m] = x[m] + b[m] * dt + noise * sq;
      if (axis_periodic(g, m)) {
        /* wrap into [lo, hi): the axis has no exit */
        double L = g->hi[m] - g->lo[m];
        double r = fmod(z[m] - g->lo[m], L);
        if (r < 0.0) r += L;
        z[m] = g->lo[m] + r;
      } else if (z[m] < g->lo[m] || z[m] > g->hi[m]) {
        int up = z[m] > g->hi[m];
        int rule = face_rule(family, m, up);
        if (rule == FACE_REFLECT) {
          /* mirror image in the face (once; the step is far shorter than the box) */
          z[m] = up ? 2.0 * g->hi[m] - z[m] : 2.0 * g->lo[m] - z[m];
        } else {
          outside = 1;
          if (rule == FACE_EXIT1) exit_one = 1;
        }
      }
    }
    /* an exit takes its face's value; value 1 wins when a point leaves
     * through several faces at once */
    double val = outside ? (exit_one ? 1.0 : 0.0) : interpolate(g, u, du, z);
    sum += wq * val;
  }
  return sum;
}

/* ------------------------------------------------------------ public --- */

/*
 * Backward march of Scheme 1 from u^{n_from} (u_in) to u^{n_to} (u_out),
 * n_to < n_from, coefficients at t_n = n dt.  boundary_rule = 1 holds the
 * boundary nodes at 1 (the Dirichlet condition of Eq. (e3)); 0 is a test
 * hook that treats boundary nodes like interior ones.  Returns 0 on success.
 */
int fko_march(const fko_grid *g, int family, const double *p, int nq,
              const double *a, const double *w, double dt, int n_from,
              int n_to, const double *u_in, double *u_out, int nthreads,
              int boundary_rule) {
  if (grid_check(g) || family_check(family, g->dim, p)) return 1;
  if (nq < 1 || !(dt > 0.0) || n_to > n_from || n_to < 0) return 1;
  int64_t J = grid_size(g);
  double *cur = (double *)malloc(sizeof(double) * J);
  double *nxt = (double *)malloc(sizeof(double) * J);
  double *du = (double *)malloc(sizeof(double) * J * g->dim);
  if (!cur || !nxt || !du) {
    free(cur); free(nxt); free(du);
    return 2;
  }
  memcpy(cur, u_in, sizeof(double) * J);
  for (int n = n_from - 1; n >= n_to; --n) {
    double tn = (double)n * dt;
    fko_slopes(g, cur, du);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t j = 0; j < J; ++j) {
      int idx[FKO_MAXDIM];
      grid_unflatten(g, j, idx);
      grid_canonical(g, idx);
      double bv = boundary_rule ? boundary_value(g, family, idx) : -1.0;
      if (bv >= 0.0)
        nxt[j] = bv;
      else
        nxt[j] = node_update(g, family, p, nq, a, w, dt, tn, cur, du, idx);
    }
    double *t = cur; cur = nxt; nxt = t;
  }
  memcpy(u_out, cur, sizeof(double) * J);
  free(cur); free(nxt); free(du);
  (void)nthreads;
  return 0;
}

/*
 * One step n (u^{n+1} -> u^n) evaluated only at the listed nodes; used to
 * check sampled outputs of very large grids.
 */
int fko_step_nodes(const fko_grid *g, int family, const double *p, int nq,
                   const double *a, const double *w, double dt, int n,
                   const double *u_next, int64_t count, const int64_t *nodes,
                   double *out, int nthreads, int boundary_rule) {
  if (grid_check(g) || family_check(family, g->dim, p)) return 1;
  int64_t J = grid_size(g);
  double *du = (double *)malloc(sizeof(double) * J * g->dim);
  if (!du) return 2;
  fko_slopes(g, u_next, du);
  double tn = (double)n * dt;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t k = 0; k < count; ++k) {
    int idx[FKO_MAXDIM];
    grid_unflatten(g, nodes[k], idx);
    grid_canonical(g, idx);
    double bv = boundary_rule ? boundary_value(g, family, idx) : -1.0;
    if (bv >= 0.0)
      out[k] = bv;
    else
      out[k] = node_update(g, family, p, nq, a, w, dt, tn, u_next, du, idx);
  }
  free(du);
  (void)nthreads;
  return 0;
}

/* The interpolant of Eq. (Lag11) alone, at points inside the closed box. */
int fko_interp(const fko_grid *g, const double *u, int64_t npts,
               const double *pts, double *out) {
  if (grid_check(g)) return 1;
  int64_t J = grid_size(g);
  double *du = (double *)malloc(sizeof(double) * J * g->dim);
  if (!du) return 2;
  fko_slopes(g, u, du);
  for (int64_t k = 0; k < npts; ++k)
    out[k] = interpolate(g, u, du, pts + k * g->dim);
  free(du);
  return 0;
}

int fko_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* ------------------------------------------------------------- adjoint --- */

/*
 * Reverse-mode derivative of the march above, for the scalar
 * L = sum_j g_j u^0_j (g = cot_u0).  Each step S_n maps u^{n+1} to u^n
 * through the slopes F (Eq. (e300)), the interpolant at the shifted points
 * (Eq. (Lag11), (e31)) and the quadrature (Eq. (e304)); its transpose is
 * applied query by query:
 *   lambda^{n+1} = (dS_n/du^{n+1})^T lambda^n,
 *   dL/dtheta   += lambda^n . dS_n/dtheta,
 * with dS_n/dtheta through the shifted points z = x + b dt + sigma
 * sqrt(2 dt) a (the exit set changes only on a null set and contributes
 * nothing), and dS_n/du through the value/derivative basis and the chain
 * rule of the slope rule (derivative of the active branch; 0 on the zero
 * branch, also when a difference is exactly 0).  Boundary rows (u = 1 for
 * n < N) depend on nothing.  theta = p[0..3] of the family: for the
 * cellular flow (A, eps, omega, D), for constant drift (b_1, b_2, b_3, s).
 * All u^n are kept in memory (test sizes only).  Single-threaded.
 */

/* d b / d theta_k (dim entries per k, k < 4) and d sigma / d theta_k */
static void drift_derivs(int family, const double *p, int dim, double t,
                         const double *x, double db[4][FKO_MAXDIM], double ds[4]) {
  for (int k = 0; k < 4; ++k) {
    ds[k] = 0.0;
    for (int m = 0; m < FKO_MAXDIM; ++m) db[k][m] = 0.0;
  }
  if (family == FKO_CONST_DRIFT) {
    for (int m = 0; m < dim; ++m) db[m][m] = 1.0;
    ds[3] = 1.0;
    return;
  }
  {
    double eps = p[1], omega = p[2], D = p[3];
    double f = sin(omega * t), df = t * cos(omega * t); /* d f / d omega */
    double X = x[0], Y = x[1];
    double cy = cos(FKO_PI * Y), sy = sin(FKO_PI * Y);
    /* b_x = -pi cos(pi y) (A sin(pi x) + eps f sin(2 pi x)) */
    /* b_y =  pi sin(pi y) (A cos(pi x) + 2 eps f cos(2 pi x)) */
    db[0][0] = -FKO_PI * cy * sin(FKO_PI * X);
    db[0][1] = FKO_PI * sy * cos(FKO_PI * X);
    db[1][0] = -FKO_PI * cy * f * sin(2.0 * FKO_PI * X);
    db[1][1] = FKO_PI * sy * 2.0 * f * cos(2.0 * FKO_PI * X);
    db[2][0] = -FKO_PI * cy * eps * df * sin(2.0 * FKO_PI * X);
    db[2][1] = FKO_PI * sy * 2.0 * eps * df * cos(2.0 * FKO_PI * X);
    ds[3] = 1.0 / sqrt(2.0 * D); /* sigma = sqrt(2 D) */
  }
}

/* derivatives of the four cell basis functions with respect to s */
static void hermite_basis_ds(double s, double h, double *dphi0, double *dphi1,
                             double *dpsi0, double *dpsi1) {
  double h3 = h * h * h, h2 = h * h;
  *dphi0 = (-6.0 * h * s + 6.0 * s * s) / h3;
  *dphi1 = (6.0 * h * s - 6.0 * s * s) / h3;
  *dpsi0 = (s - h) * (3.0 * s - h) / h2;
  *dpsi1 = s * (3.0 * s - 2.0 * h) / h2;
}

/* partial derivatives of the PCHIP rule 2/(1/dl + 1/dr) (0 off its branch) */
static void pchip_rule_grad(double dl, double dr, double *gl, double *gr) {
  if (dl * dr <= 0.0) {
    *gl = 0.0;
    *gr = 0.0;
    return;
  }
  double s = dl + dr;
  *gl = 2.0 * dr * dr / (s * s);
  *gr = 2.0 * dl * dl / (s * s);
}

/* lam_u[i] += sum_j mu[j] d(slope_j)/d u_i along axis m (transpose of F) */
static void slopes_axis_transpose(const fko_grid *g, int m, const double *u,
                                  const double *mu, double *lam_u) {
  int64_t J = grid_size(g);
  int64_t st = grid_stride(g, m);
  int nm = g->n[m];
  double h = grid_h(g, m);
  int idx[FKO_MAXDIM];
  for (int64_t j = 0; j < J; ++j) {
    if (mu[j] == 0.0) continue;
    grid_unflatten(g, j, idx);
    int i = idx[m];
    int64_t base = j - (int64_t)i * st;
    /* the two differences used at node i, as (upper, lower) node pairs */
    int l1, l0, r1, r0;
    if (i == 0) {
      l1 = 1; l0 = 0; r1 = 2; r0 = 1;
    } else if (i == nm - 1) {
      l1 = nm - 1; l0 = nm - 2; r1 = nm - 2; r0 = nm - 3;
    } else {
      l1 = i; l0 = i - 1; r1 = i + 1; r0 = i;
    }
    double dl = (u[base + (int64_t)l1 * st] - u[base + (int64_t)l0 * st]) / h;
    double dr = (u[base + (int64_t)r1 * st] - u[base + (int64_t)r0 * st]) / h;
    double gl, gr;
    pchip_rule_grad(dl, dr, &gl, &gr);
    lam_u[base + (int64_t)l1 * st] += mu[j] * gl / h;
    lam_u[base + (int64_t)l0 * st] -= mu[j] * gl / h;
    lam_u[base + (int64_t)r1 * st] += mu[j] * gr / h;
    lam_u[base + (int64_t)r0 * st] -= mu[j] * gr / h;
  }
}

int fko_adjoint(const fko_grid *g, int family, const double *p, int nq,
                const double *a, const double *w, double dt, int n_steps,
                const double *u_terminal, const double *cot_u0,
                double *dtheta, double *du_terminal) {
  if (grid_check(g) || family_check(family, g->dim, p)) return 1;
  if (nq < 1 || !(dt > 0.0) || n_steps < 1) return 1;
  if (g->periodic || family == FKO_PAPER_CELLULAR || family == FKO_RUNAWAY ||
      family == FKO_RUNAWAY_QUENCH)
    return 3; /* not differentiated */
  for (int m = 0; m < g->dim; ++m)
    if (g->axis[m]) return 3; /* uniform meshes only */
  int d = g->dim;
  int64_t J = grid_size(g);
  double *us = (double *)malloc(sizeof(double) * J * (size_t)(n_steps + 1));
  double *du = (double *)malloc(sizeof(double) * J * d);
  double *lam = (double *)malloc(sizeof(double) * J);
  double *lam_next = (double *)malloc(sizeof(double) * J);
  double *mu_u = (double *)malloc(sizeof(double) * J);
  double *mu_d = (double *)malloc(sizeof(double) * J * d);
  if (!us || !du || !lam || !lam_next || !mu_u || !mu_d) {
    free(us); free(du); free(lam); free(lam_next); free(mu_u); free(mu_d);
    return 2;
  }
  /* forward: us + n J holds u^n */
  memcpy(us + (int64_t)n_steps * J, u_terminal, sizeof(double) * J);
  for (int n = n_steps - 1; n >= 0; --n)
    fko_march(g, family, p, nq, a, w, dt, n + 1, n, us + (int64_t)(n + 1) * J,
              us + (int64_t)n * J, 1, 1);
  for (int k = 0; k < 4; ++k) dtheta[k] = 0.0;
  memcpy(lam, cot_u0, sizeof(double) * J);
  double sq = sqrt(2.0 * dt);
  int64_t nqd = 1;
  for (int m = 0; m < d; ++m) nqd *= nq;
  for (int n = 0; n < n_steps; ++n) {
    const double *u = us + (int64_t)(n + 1) * J; /* input of step n */
    double tn = (double)n * dt;
    fko_slopes(g, u, du);
    memset(mu_u, 0, sizeof(double) * J);
    memset(mu_d, 0, sizeof(double) * J * d);
    for (int64_t j = 0; j < J; ++j) {
      int idx[FKO_MAXDIM];
      grid_unflatten(g, j, idx);
      if (boundary_value(g, family, idx) >= 0.0 || lam[j] == 0.0) continue;
      double x[FKO_MAXDIM], b[FKO_MAXDIM], sig[FKO_MAXDIM * FKO_MAXDIM];
      double db[4][FKO_MAXDIM], ds[4];
      for (int m = 0; m < d; ++m) x[m] = grid_x(g, m, idx[m]);
      fko_coefficients(family, p, d, tn, x, b, sig);
      drift_derivs(family, p, d, tn, x, db, ds);
      for (int64_t qq = 0; qq < nqd; ++qq) {
        int q[FKO_MAXDIM];
        int64_t r = qq;
        double wq = 1.0;
        for (int m = 0; m < d; ++m) {
          q[m] = (int)(r % nq);
          r /= nq;
          wq *= w[q[m]];
        }
        double z[FKO_MAXDIM];
        int outside = 0;
        for (int m = 0; m < d; ++m) {
          double noise = 0.0;
          for (int k = 0; k < d; ++k) noise += sig[m * d + k] * a[q[k]];
          z[m] = x[m] + b[m] * dt + noise * sq;
          if (z[m] < g->lo[m] || z[m] > g->hi[m]) outside = 1;
        }
        if (outside) continue; /* the exit value 1 depends on nothing */
        double W = lam[j] * wq;
        int c[FKO_MAXDIM];
        double phi[FKO_MAXDIM][2], psi[FKO_MAXDIM][2];
        double dphi[FKO_MAXDIM][2], dpsi[FKO_MAXDIM][2];
        for (int m = 0; m < d; ++m) {
          double h = grid_h(g, m);
          int cm = (int)floor((z[m] - g->lo[m]) / h);
          if (cm < 0) cm = 0;
          if (cm > g->n[m] - 2) cm = g->n[m] - 2;
          c[m] = cm;
          double s = z[m] - grid_x(g, m, cm);
          hermite_basis(s, h, &phi[m][0], &phi[m][1], &psi[m][0], &psi[m][1]);
          hermite_basis_ds(s, h, &dphi[m][0], &dphi[m][1], &dpsi[m][0], &dpsi[m][1]);
        }
        double grad[FKO_MAXDIM] = {0.0, 0.0, 0.0}; /* d Itilde / d z_m */
        for (int corner = 0; corner < (1 << d); ++corner) {
          int64_t node = 0;
          for (int m = 0; m < d; ++m)
            node += (int64_t)(c[m] + ((corner >> m) & 1)) * grid_stride(g, m);
          /* value term */
          double wv = 1.0;
          for (int m = 0; m < d; ++m) wv *= phi[m][(corner >> m) & 1];
          mu_u[node] += W * wv;
          for (int k = 0; k < d; ++k) {
            double gv = 1.0;
            for (int m = 0; m < d; ++m) {
              int bit = (corner >> m) & 1;
              gv *= (m == k) ? dphi[m][bit] : phi[m][bit];
            }
            grad[k] += gv * u[node];
          }
          /* derivative terms */
          for (int m = 0; m < d; ++m) {
            double wd = 1.0;
            for (int k = 0; k < d; ++k) {
              int bit = (corner >> k) & 1;
              wd *= (k == m) ? psi[k][bit] : phi[k][bit];
            }
            mu_d[(int64_t)m * J + node] += W * wd;
            for (int kk = 0; kk < d; ++kk) {
              double gd = 1.0;
              for (int k = 0; k < d; ++k) {
                int bit = (corner >> k) & 1;
                double f;
                if (k == m)
                  f = (k == kk) ? dpsi[k][bit] : psi[k][bit];
                else
                  f = (k == kk) ? dphi[k][bit] : phi[k][bit];
                gd *= f;
              }
              grad[kk] += gd * du[(int64_t)m * J + node];
            }
          }
        }
        /* dz_m / dtheta_k = db_k,m dt + dsigma_k sqrt(2 dt) (sigma-scaled noise) */
        for (int k = 0; k < 4; ++k) {
          double dz = 0.0;
          for (int m = 0; m < d; ++m) {
            double noise_m = 0.0;
            for (int kk = 0; kk < d; ++kk) noise_m += (kk == m ? 1.0 : 0.0) * a[q[kk]];
            dz += grad[m] * (db[k][m] * dt + ds[k] * noise_m * sq);
          }
          dtheta[k] += W * dz;
        }
      }
    }
    /* lambda^{n+1} = mu_u + F^T mu_d */
    memcpy(lam_next, mu_u, sizeof(double) * J);
    for (int m = 0; m < d; ++m) slopes_axis_transpose(g, m, u, mu_d + (int64_t)m * J, lam_next);
    double *t = lam; lam = lam_next; lam_next = t;
  }
  memcpy(du_terminal, lam, sizeof(double) * J);
  free(us); free(du); free(lam); free(lam_next); free(mu_u); free(mu_d);
  return 0;
}
