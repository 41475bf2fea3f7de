/*
 * fk.h -- C ABI of a GB300 (sm_103a) library for the Feynman-Kac backward
 * march that computes exit-time probabilities of SDEs (Yang, Zhang,
 * del-Castillo-Negrete, Stoyanov, "A Feynman-Kac based numerical method for
 * the exit time probability of a class of transport problems",
 * arXiv 2104.14561).
 *
 * The method (Sec. 3.1, Scheme 1).  For the SDE dX = b(t,X) dt +
 * sigma(t,X) dW (Eq. (e1)) in an open box D (Sec. 2), the exit probability
 * P(T,x) = u(0,x) (Eq. (e5)) is approximated on a Cartesian mesh S by
 * marching backward from the terminal field u^N, n = N-1, ..., 0:
 *
 *   u^n_j = sum_q w_q Itilde[u^{n+1}](x_j + b(t_n,x_j) dt
 *                                      + sigma(t_n,x_j) sqrt(2 dt) a_q)
 *
 * with the tensor Gauss-Hermite rule (a_q, w_q) of Eq. (quad) normalised to
 * the density pi^{-d/2} exp(-|xi|^2) of Eq. (expec), the piecewise cubic
 * Hermite interpolant Itilde of Eq. (Lag11) whose nodal derivatives follow
 * the PCHIP rule Eq. (e300), the exit value 1 for a shifted point outside
 * the closed box (Eq. (e24)), and boundary nodes held at 1 (Eq. (e3)).
 *
 * Conventions for every call:
 *  - Fields are dense arrays of the plan's precision (float for FK_FP32,
 *    double for FK_FP64) with one value per mesh node, x fastest:
 *    u[(k * n[1] + j) * n[0] + i] for node (i, j, k).  Node i on axis m sits
 *    at lo[m] + i * (hi[m] - lo[m]) / (n[m] - 1).
 *  - "Device pointer" means memory of the plan's CUDA device (cudaMalloc,
 *    a PyTorch CUDA tensor, ...).  The caller owns every buffer it passes;
 *    the library never frees or retains caller memory after a call returns.
 *  - Calls that take a cudaStream_t are asynchronous on that stream; they
 *    return after enqueueing.  A plan must not be used from two host
 *    threads at once.
 *  - Every call returns an fk_status; no C++ exception crosses the ABI.
 *    Arguments are validated before any CUDA call is made.
 */
#ifndef FK_H
#define FK_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fk_status {
  FK_OK = 0,
  FK_ERR_INVALID_ARG = 1, /* a NULL, out-of-range or inconsistent argument */
  FK_ERR_UNSUPPORTED = 2, /* valid, but not a case the library implements */
  FK_ERR_OOM = 3,         /* device allocation failed                     */
  FK_ERR_CUDA = 4,        /* a CUDA runtime call failed                   */
  FK_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up           */
  FK_ERR_DEVICE = 6       /* a device-side range check fired              */
} fk_status;

typedef enum fk_precision { FK_FP32 = 0, FK_FP64 = 1 } fk_precision;

/* FK_PATH_MATRIX_FREE recomputes shifted points and interpolation weights
 * in every step (one fused kernel per step).  FK_PATH_CSR assembles the
 * product Q Psi of Eq. (e36) once as a sparse matrix and applies it every
 * step; it needs coefficients that do not depend on t. */
typedef enum fk_path { FK_PATH_MATRIX_FREE = 0, FK_PATH_CSR = 1 } fk_path;

/* Coefficient families (b, sigma of Eq. (e1)):
 *  FK_CONST_DRIFT     p = {b_1, b_2, b_3, s}: b constant, sigma = s I
 *                     (Sec. 4.1 is d = 1, b = 0, s = 1).  d = 1, 2 or 3
 *                     (the only family with d = 3).
 *  FK_CELLULAR_FLOW   p = {A, eps, omega, D}, d = 2: the time-periodic
 *                     cellular flow of Sec. 4.2 written with the stream
 *                     function psi = A sin(pi x) sin(pi y)
 *                       + eps sin(omega t) sin(2 pi x) sin(pi y),
 *                     b = (-d psi/dy, d psi/dx), sigma = sqrt(2 D) I.
 *  FK_PAPER_CELLULAR  p = {Pe, n, eps, omega}, d = 2: the paper's own
 *                     example of Sec. 4.2, dx = Pe v dt + dW, with
 *                       v_1 = -pi cos(pi x_2)[sin(n x_1) + eps f cos(n x_1)],
 *                       v_2 =  n sin(pi x_2)[cos(n x_1) - eps f sin(n x_1)],
 *                     f = cos(omega t), sigma = I.  Usually with the region
 *                     FK_PERIODIC_X on [-pi, pi] x [0, 1].  Matrix-free
 *                     path only; fk_adjoint returns FK_ERR_UNSUPPORTED.
 *  FK_RUNAWAY_3D      d = 3, x = (p, xi, r): the runaway-electron model of
 *                     Sec. 4.3, Eq. (ex32d), with
 *                     p = {E, tau, Z, delta, nu_ee, v_T, r_D, W, Delta_p,
 *                          V_0, D_0} (the paper's values: 0.3, 1e5, 1,
 *                     0.042, 1, 1, 0.7, 1e-2, 20, 0.003, 1e-4).  The box is
 *                     [p_min, p_max] x [xi_lo, xi_hi] x [r_lo, r_hi] with
 *                     p_min > 0, -1 <= xi_lo < xi_hi <= 1, r_lo >= 0.  The
 *                     faces act as follows (the region must be
 *                     FK_ALL_FACES_ABSORBING; this family fixes them): an
 *                     exit through p = p_max takes 1 (runaway), through
 *                     p = p_min or r = r_hi (the wall) 0, and the faces of
 *                     xi and r = r_lo mirror a shifted point back into the
 *                     box; nodes on those faces are updated, nodes on the
 *                     absorbing faces hold their value (1 on p = p_max).
 *                     The terminal indicator is 1 on p = p_max only.
 *                     Uniform mesh, matrix-free; fk_adjoint, batching and
 *                     the static entry return FK_ERR_UNSUPPORTED.
 *  FK_RUNAWAY_QUENCH_3D  the time-dependent variant at the end of Sec. 4.3
 *                     (a thermal quench), p = {E_0, tau, Z, T0, Tf, Ttilde,
 *                     t_star, r_D, W, Delta_p, V_0, D_0, mc2}; at time t the
 *                     FK_RUNAWAY_3D model runs with the constants that
 *                     fk_runaway_quench_params returns for t (the paper's
 *                     values: 1e-3, 6000, 1, 3, 0.005, 3, t_star, 0, 1e-4,
 *                     2, 0, D_0, with temperatures in keV and mc2 = 511).
 *                     Same box, faces and restrictions as FK_RUNAWAY_3D;
 *                     T0, Tf, Ttilde, t_star and mc2 must be positive and
 *                     ln Lambda(T) positive at T0, Tf and Ttilde
 *                     (FK_ERR_INVALID_ARG).  Plan creation evaluates the
 *                     coefficients at every time step to bound the window. */
enum {
  FK_CONST_DRIFT = 0,
  FK_CELLULAR_FLOW = 1,
  FK_PAPER_CELLULAR = 2,
  FK_RUNAWAY_3D = 3,
  FK_RUNAWAY_QUENCH_3D = 4
};

/* Cartesian mesh S (Sec. 3.1.2): n[m] >= 3 nodes on [lo[m], hi[m]] for
 * m < dim; entries for m >= dim are ignored.  axis[m] = NULL gives the
 * uniform mesh; otherwise it points to n[m] strictly increasing host
 * coordinates with axis[m][0] = lo[m] and axis[m][n[m]-1] = hi[m] (the
 * partition along a direction need not be uniform), read during plan
 * creation only.  Non-uniform axes: d = 1 or 2, FK_PATH_MATRIX_FREE, every
 * face absorbing; Eq. (e300) then takes divided differences over the actual
 * spacings and the Hermite cell formula each cell's own width. */
typedef struct fk_grid {
  int dim;
  int n[3];
  double lo[3];
  double hi[3];
  const double *axis[3];
} fk_grid;

/* Which faces of the box absorb (exit value 1).  Bit 2m is the lower face
 * of axis m, bit 2m+1 the upper face.  Two masks are implemented:
 *  FK_ALL_FACES_ABSORBING  every face absorbs;
 *  FK_PERIODIC_X           (d = 2, matrix-free path) the two x faces are
 *                          identified instead: node n[0]-1 is node 0, the
 *                          period is n[0] - 1 nodes, slopes and shifted
 *                          points wrap around in x and nothing exits
 *                          through x; the y faces absorb (Sec. 4.2's
 *                          example).  The terminal indicator is then 1 on
 *                          the y faces only, and fields must hold equal
 *                          values in columns 0 and n[0]-1.
 * Any other mask gives FK_ERR_UNSUPPORTED. */
typedef struct fk_region {
  unsigned absorbing_faces;
} fk_region;
#define FK_ALL_FACES_ABSORBING 0x3Fu
#define FK_PERIODIC_X 0x3Cu

typedef struct fk_coeffs {
  int family;
  double p[16];   /* family parameters; unused entries are ignored but must be finite */
} fk_coeffs;

typedef struct fk_plan fk_plan;

/* Read-only description of a plan (fk_plan_get_info). */
typedef struct fk_plan_info {
  int64_t n_nodes;          /* J                                        */
  int64_t n_interior;       /* nodes strictly inside the box            */
  int dim, q_per_dim, n_steps, precision, path;
  int halo[3];              /* halo of a tile, in cells, per axis       */
  int tile[3];              /* output nodes per tile, per axis          */
  double reach_cells[3];    /* bound on |shift| in cells, per axis      */
  int64_t csr_nnz;          /* stored entries of Q Psi (FK_PATH_CSR)    */
  int64_t workspace_bytes;  /* device memory owned by the plan          */
  int window_rows;          /* 2D FP32 step kernel: width W of its node
                               window (0 = the direct kernel)            */
  int step_kernel;          /* 2D step kernel in use: 0 direct (per-point
                               Hermite evaluation), 1 row window (y-rows
                               read once per x-point, direct face bands),
                               2 masked tensor window (W x W nodes per
                               node, exits as zero weights); 1D: 0 one
                               launch per step, 3 the whole march in one
                               CTA's shared memory, 4 in one thread-block
                               cluster (distributed shared memory); 3D:
                               5, the node-window kernel (W^3 records
                               per node, exits as zero weights)          */
  int batch_mode;           /* strategy of the last fk_solve_batched this
                               plan led (plans[0]): 0 none, 1 the
                               persistent kernel, 2 concurrent single-plan
                               graphs on side streams                    */
  int adjoint_kernel;       /* backward step of the last fk_adjoint: 0 none
                               yet, 1 per-point transposed scatter, 2 masked
                               tensor window                             */
  int periodic_x;           /* 1: region FK_PERIODIC_X                   */
  int nonuniform;           /* 1: some axis has explicit coordinates     */
  int march_mode;           /* whole marches without snapshots: 0 one
                               launch per step, 1 one persistent launch
                               for every step (2D FP32 masked kernel:
                               tiles wait on their 3 x 3 neighbourhood's
                               step counters, chosen at plan creation
                               when a timed 16-step march is faster)     */
  int nodes_per_thread;     /* 2D FP32 masked kernel: 1, or 2 when each
                               thread takes two nodes of a column and
                               reads the rows their windows share once
                               (W = 7; chosen by the timing at plan
                               creation); 1 for every other kernel       */
} fk_plan_info;

/* ------------------------------------------------------------------------
 * fk_plan_create -- validate a problem and prepare everything a march needs.
 * Problem statement: Eq. (e1) (b, sigma), Sec. 2 (the box D), Sec. 3.1.2
 * (mesh S), Eq. (quad) (q_per_dim Gauss-Hermite points per axis, so Q =
 * q_per_dim^dim shifted points per node), Sec. 3.1.1 (uniform time step dt,
 * N = n_steps steps, T = N dt, coefficients evaluated at t_n = n dt).
 *   out        receives the new plan (set to NULL on failure).
 *   q_per_dim  1..8 for dim = 2 or 3, 1..16 for dim = 1.
 *   dt > 0, n_steps >= 1.
 *   path       FK_PATH_CSR needs a family whose coefficients do not depend
 *              on t (FK_CONST_DRIFT, or FK_CELLULAR_FLOW with eps = 0),
 *              else FK_ERR_UNSUPPORTED.
 *   dim = 3    FK_CONST_DRIFT or FK_RUNAWAY_3D on a uniform mesh (axis[]
 *              NULL), FK_ALL_FACES_ABSORBING, FK_PATH_MATRIX_FREE,
 *              n[m] <= 65535.  The node window W must be at most 8 and at
 *              most every n[m]: W = floor(span) + 3 with span the largest
 *              sigma_m sqrt(2 dt) (a_{q-1} - a_0) / h_m over the nodes (for
 *              the runaway model also at least floor(|b_m| dt / h_m +
 *              span / 2) + 2, so that mirrored points stay in the window);
 *              else FK_ERR_UNSUPPORTED.
 *              fk_solve_batched, fk_adjoint and fk_solve_static take
 *              dim = 2 plans only (FK_ERR_UNSUPPORTED).
 * The plan allocates its own device workspace on the current CUDA device
 * (coefficient tables, one scratch field, for FK_PATH_CSR the assembled
 * matrix, which is built here).  Errors: FK_ERR_INVALID_ARG,
 * FK_ERR_UNSUPPORTED, FK_ERR_OOM, FK_ERR_CUDA.
 * ---------------------------------------------------------------------- */
fk_status fk_plan_create(fk_plan **out, const fk_grid *grid,
                         const fk_region *region, const fk_coeffs *coeffs,
                         int q_per_dim, double dt, int n_steps,
                         fk_precision prec, fk_path path);

/* Release a plan and all device memory it owns (NULL is a no-op).  Waits
 * for the plan's own work to finish. */
fk_status fk_plan_destroy(fk_plan *plan);

/* Copy the plan's description into *info. */
fk_status fk_plan_get_info(const fk_plan *plan, fk_plan_info *info);

/* ------------------------------------------------------------------------
 * fk_gauss_hermite -- the 1D rule the plans use: q nodes a[] (ascending) and
 * weights w[] for the density pi^{-1/2} exp(-xi^2) of Eq. (expec), so that
 * sum w = 1.  Host arrays of length q, 1 <= q <= 16.  Host-only call.
 * ---------------------------------------------------------------------- */
fk_status fk_gauss_hermite(int q, double *a, double *w);

/* ------------------------------------------------------------------------
 * fk_runaway_quench_params -- the constants of the runaway model at time t
 * of the thermal-quench variant (end of Sec. 4.3): with
 *   T(t) = Tf + (T0 - Tf) exp(-t / t_star),
 *   ln Lambda(T) = 14.9 - (1/2) ln 0.28 + ln T,
 * it writes p11 = {E_0 (T0/T)^{3/2}, tau, Z, sqrt(2 T / mc2),
 * (Ttilde/T)^{3/2} ln Lambda(T) / ln Lambda(Ttilde), sqrt(T / Ttilde), r_D,
 * W, Delta_p, V_0, D_0}, the FK_RUNAWAY_3D parameter block.
 *   p13  host array of the 13 FK_RUNAWAY_QUENCH_3D parameters.
 *   t    time.
 *   p11  host array of 11 doubles, written.
 * Host-only call.  FK_ERR_INVALID_ARG for NULL pointers, a non-finite t, or
 * T0, Tf, Ttilde, t_star or mc2 not positive.
 * ---------------------------------------------------------------------- */
fk_status fk_runaway_quench_params(const double *p13, double t, double *p11);

/* ------------------------------------------------------------------------
 * fk_solve -- Scheme 1 from n = N to n = 0: u_out <- u^0 = P(T, x_j).
 *   u_terminal  device pointer to u^N, or NULL for the terminal indicator
 *               chi of Sec. 3.2 (0 inside, 1 on the boundary).  Read only.
 *               May equal u_out.
 *   u_out       device pointer, receives u^0.
 *   snapshots   NULL, or a device buffer of floor(N / snapshot_stride)
 *               fields: field m receives u^{N - (m+1) snapshot_stride}.
 *               For coefficients that do not depend on t this is
 *               P((m+1) snapshot_stride dt, x): the whole time history
 *               (Sec. 3.2) from one march.
 *   stream      CUDA stream; the march is enqueued as one CUDA graph.
 * ---------------------------------------------------------------------- */
fk_status fk_solve(fk_plan *plan, const void *u_terminal, void *u_out,
                   void *snapshots, int snapshot_stride, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * fk_solve_host -- fk_solve (Scheme 1, Sec. 3.1.5) with the fields in host
 * memory: copies u^N to the device, runs the march, copies u^0 back, all
 * enqueued on `stream` in that order.
 *   u_terminal_host  host pointer to u^N (J values of the plan's precision,
 *                    laid out as fk_solve's fields), or NULL for the
 *                    terminal indicator chi.  Read only.
 *   u_out_host       host pointer, receives u^0 (J values).  May equal
 *                    u_terminal_host.
 *   stream           CUDA stream.  The call returns once the work is
 *                    enqueued: u_out_host holds u^0 when the stream has
 *                    passed it (cudaStreamSynchronize).  With page-locked
 *                    buffers (cudaHostAlloc, cudaHostRegister) the copies
 *                    are asynchronous; pageable buffers are staged by the
 *                    CUDA driver and can block the calling thread.
 * The device copy of the field is one plan-owned buffer of J values,
 * allocated on the first call (FK_ERR_OOM if that fails; counted in
 * workspace_bytes) and freed with the plan.  Calls on one plan whose work
 * overlaps on the GPU share that buffer and race.
 * ---------------------------------------------------------------------- */
fk_status fk_solve_host(fk_plan *plan, const void *u_terminal_host, void *u_out_host,
                        cudaStream_t stream);

/* ------------------------------------------------------------------------
 * fk_march -- the steps n = n_from-1, ..., n_to of Scheme 1 only:
 * u_out <- u^{n_to} given u_in = u^{n_from}, 0 <= n_to <= n_from <= N.
 * The march is Markov in (n, u^n), so this is also checkpoint / resume.
 * u_in may equal u_out.  Device pointers.  n_to == n_from copies.
 * ---------------------------------------------------------------------- */
fk_status fk_march(fk_plan *plan, int n_from, int n_to, const void *u_in,
                   void *u_out, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * fk_solve_horizons -- Algorithm 1 of Sec. 3.2: P(t_k, x_j) for every
 * horizon t_k = k dt, k = 1..N, in one backward pass.  Horizon k is the
 * march of Scheme 1 over k steps with the coefficients of times
 * t_{k-1}, ..., t_0 (start at time 0, exit by t_k), so for coefficients
 * that depend on t each horizon is a separate march; the pass updates all
 * horizons that are still active at step n with one launch.  Work is
 * N (N + 1) / 2 single-field steps.  (For coefficients that do not depend
 * on t, fk_solve's snapshots give the same history from one march.)
 *   u_terminal  device pointer to the terminal field (J values) shared by
 *               all horizons, or NULL for the indicator chi.  Read only; it
 *               must not overlap p_out.
 *   p_out       device buffer of N fields of J values (the plan's precision);
 *               field k - 1 receives P(t_k, .).
 *   stream      CUDA stream; N launches are enqueued.
 * The plan allocates a second buffer of N fields on first use (grown on
 * demand, freed with the plan).  Errors: FK_ERR_INVALID_ARG,
 * FK_ERR_UNSUPPORTED (FK_PATH_CSR plans), FK_ERR_OOM, FK_ERR_CUDA.
 * ---------------------------------------------------------------------- */
fk_status fk_solve_horizons(fk_plan *plan, const void *u_terminal, void *p_out,
                            cudaStream_t stream);

/* ------------------------------------------------------------------------
 * fk_solve_batched -- fk_solve for n independent plans (same precision,
 * dim = 2, FK_PATH_MATRIX_FREE, same q_per_dim and n_steps) in ONE
 * persistent kernel: the tiles of every instance share one work list and
 * the steps are separated by a bounded grid barrier (Sec. 5 of the paper's
 * conclusion notes that batches parallelise directly).
 *   plans[i], u_terminal[i] (NULL = chi), u_out[i] (device) per instance.
 * Returns FK_ERR_TIMEOUT (after the kernel has stopped) if a device-side
 * barrier wait exceeded its bound.
 * ---------------------------------------------------------------------- */
fk_status fk_solve_batched(int n, fk_plan *const *plans,
                           const void *const *u_terminal, void *const *u_out,
                           cudaStream_t stream);

/* ------------------------------------------------------------------------
 * fk_adjoint -- reverse-mode derivative of the scalar L = <g, u^0>, where
 * u^0 = S_0(S_1(...S_{N-1}(u^N))) is the march and g = cotangent_u0 (FP64
 * device array, one value per node).  Each step S_n is differentiated
 * exactly: the transpose of the interpolation-and-quadrature map of
 * Eqs. (e34)-(e36) applied to [u; du], the transpose of the slope map F
 * (Eq. (e300), derivative taken on its active branch), and the derivative
 * of the shifted points of Eq. (e31) with respect to the coefficients.
 *   u_terminal      device pointer to u^N or NULL (= chi).
 *   dtheta          device FP64 array of 4 entries, receives
 *                   dL/d(p[0..3]) of the coefficient family (for
 *                   FK_CELLULAR_FLOW: A, eps, omega, D).  May be NULL.
 *   du_terminal     device array of the plan's precision, receives dL/du^N.
 *                   May be NULL.
 *   checkpoint_every K >= 1: u is stored every K steps on the forward pass
 *                   and each segment is recomputed in reverse.
 * Only dim = 2, FK_PATH_MATRIX_FREE plans.  Gradients are accumulated in
 * FP64 whatever the march precision.
 * ---------------------------------------------------------------------- */
fk_status fk_adjoint(fk_plan *plan, const void *u_terminal,
                     const double *cotangent_u0, double *dtheta,
                     void *du_terminal, int checkpoint_every,
                     cudaStream_t stream);

/* fk_adjoint_kernel_times -- a measurement aid (no counterpart in the
 * paper).  With record = 1, later fk_adjoint calls on this plan record a
 * CUDA event on their stream right before and right after each launch of
 * the backward-step kernel (the transposed step; the slope transpose that
 * follows it is outside the pair); with record = 0 they stop.  Each call of
 * this function first waits for the events of the last recorded fk_adjoint
 * and writes their summed elapsed time (ms) to *kernel_ms and the number of
 * pairs to *launches (0 and 0 if nothing was recorded; either pointer may
 * be NULL), then sets the recording state.  The events are created by the
 * first recorded fk_adjoint (2 N of them) and freed with the plan. */
fk_status fk_adjoint_kernel_times(fk_plan *plan, int record, double *kernel_ms,
                                  int *launches);

/* Text for a status code (static storage). */
const char *fk_status_string(fk_status status);

/* Synchronise with the plan's device and report (then clear) the plan's
 * device-side error word: FK_OK, FK_ERR_DEVICE (a range check fired) or
 * FK_ERR_TIMEOUT (a bounded wait gave up). */
fk_status fk_last_device_error(fk_plan *plan);

/* ------------------------------------------------------------------------
 * fk_solve_static -- the same march as fk_solve for a 2D FK_PATH_MATRIX_FREE
 * problem, for callers that cannot allocate device memory.  The paper has no
 * counterpart; this exists only for such callers: applications whose own
 * pool allocator owns all device memory and forbids libraries from calling
 * cudaMalloc beside it, and latency-bound loops that cannot afford the
 * device-wide synchronisation of cudaMalloc / cudaFree.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine, host or
 * device.  Everything besides the caller's buffers (one scratch field, the
 * coefficient tables, an error word) lives in one static device array of
 * 16 MiB, which every GPU that loads this library holds until the process
 * exits.
 *   grid, coeffs, q_per_dim, dt, n_steps, prec  as for fk_plan_create, with
 *               grid->dim = 2 and a uniform mesh (axis[] NULL); families
 *               FK_CONST_DRIFT and FK_CELLULAR_FLOW.  There is no region
 *               argument: every face of the box absorbs.
 *   u_terminal  device pointer to u^N, or NULL for chi; may equal u_out.
 *   u_out       device pointer, receives u^0.
 * Size limit: 256 + 4 n[0] e + 2 n[1] e + n[0] n[1] e bytes (e = 4 for FP32,
 * 8 for FP64; each of the three tables rounded up to 256 B) must fit in
 * 16 MiB -- about 4.1 million nodes in FP32, 2.09 million in FP64.  Larger
 * problems get FK_ERR_INVALID_ARG before anything is enqueued.
 * A CUDA error already pending in the calling thread (from earlier work of
 * the caller) gives FK_ERR_CUDA before anything is enqueued; the error is
 * left pending for the caller.
 * The first call on each device does a one-time set-up on that device (it
 * looks up the device address of the static array and opts the step kernels
 * into large shared memory); make that first call before any stream
 * capture.  The set-up is kept for the life of the process: resetting the
 * device (cudaDeviceReset) after the first call is not supported.  Every
 * call on a device uses the same array and overwrites what the previous
 * call left there: calls whose work overlaps on the GPU (two streams, two
 * host threads) race and corrupt each other's results.
 * ---------------------------------------------------------------------- */
fk_status fk_solve_static(const fk_grid *grid, const fk_coeffs *coeffs,
                          int q_per_dim, double dt, int n_steps,
                          fk_precision prec, const void *u_terminal,
                          void *u_out, cudaStream_t stream);

/* fk_static_last_device_error -- the device error word of fk_solve_static
 * calls on the current device (like fk_last_device_error for a plan; no
 * counterpart in the paper).  It waits for all work on the current device
 * (cudaDeviceSynchronize), then reads and clears the word in the static
 * array: FK_OK, FK_ERR_DEVICE (a step kernel's range check fired: a
 * shifted point fell outside its tile's halo, and that result is wrong) or
 * FK_ERR_CUDA.  Each fk_solve_static call clears the word at the start of
 * its own work on the GPU, so the answer covers the last call.  Allocates
 * nothing; not for use during stream capture. */
fk_status fk_static_last_device_error(void);

/* ------------------------------------------------------------------------
 * fk_measure_fma_rate -- a measurement aid with no counterpart in the
 * paper: the fused multiply-add throughput of the current device, the
 * denominator of the march kernels' ALU rooflines.  Every thread slot of
 * every SM runs eight independent FMA chains from registers; the kernel is
 * timed with CUDA events on `stream` and the call waits for it.
 *   prec     FK_FP32 or FK_FP64.
 *   packed   FK_FP32 only: 1 times the packed f32x2 form (two FMAs per
 *            instruction), 0 the scalar form.
 *   seconds  target duration of the timed launch, (0, 10].
 *   flop_per_s  receives 2 x FMAs per second (0 on error).
 * Errors: FK_ERR_INVALID_ARG, FK_ERR_CUDA.  Allocates nothing.
 * ---------------------------------------------------------------------- */
fk_status fk_measure_fma_rate(fk_precision prec, int packed, double seconds,
                              double *flop_per_s, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FK_H */
