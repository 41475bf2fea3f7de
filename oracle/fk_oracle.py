"""FP64 CPU oracle for the Feynman-Kac exit-probability march (arXiv 2104.14561).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product path
(``paper_2104_14561_gb300``) never does, and this module imports nothing
from it.

Contents
--------
* ``build()`` compiles ``fk_oracle.c`` (plain C, FP64, -ffp-contract=off).
* ``gauss_hermite(q)``: the 1D Gauss-Hermite rule of Eq. (quad) normalised to
  the density pi^{-1/2} exp(-xi^2) of Eq. (expec), by Golub-Welsch (the
  eigen-decomposition of the Jacobi matrix of the orthonormal Hermite
  polynomials; numpy's symmetric eigensolver is the library step).
* ``march`` / ``step_nodes`` / ``interp`` / ``slopes`` / ``coefficients``:
  ctypes wrappers of the C statement of Scheme 1.
* ``terminal_indicator``: chi of Sec. 3.2 (0 inside, 1 on the boundary).
* ``exit_prob_1d_image`` / ``exit_prob_1d_eigen``: two independent closed
  forms of the exit probability of 1D Brownian motion with constant drift
  from an interval (Sec. 4.1 generalised to drift; Eq. (e45) is the
  driftless case with only odd terms, see ``exit_prob_1d_paper_e45``).
* ``mc_exit_prob``: Euler-Maruyama Monte Carlo with the exit checked at the
  discrete times t_n, the estimator named in the introduction (O(1/sqrt N)).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_*.py) against closed forms, textbook tables, library
routines, brute force or Monte Carlo.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fk_oracle.c")
_LIB = os.path.join(_HERE, "libfk_oracle.so")

CONST_DRIFT = 0
CELLULAR_FLOW = 1
PAPER_CELLULAR = 2   # the paper's own example of Sec. 4.2: p = (Pe, n, eps, omega), sigma = I
RUNAWAY = 3          # the runaway-electron model of Sec. 4.3 (d = 3, x = (p, xi, r)):
#                      params (E, tau, Z, delta, nu_ee, v_T, r_D, W, Delta_p, V_0, D_0)
RUNAWAY_PARAMS = (0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003, 1e-4)  # Sec. 4.3
RUNAWAY_QUENCH = 4   # the thermal-quench (time-dependent) variant, params
#                      (E_0, tau, Z, T0, Tf, Ttilde, t_star, r_D, W, Delta_p, V_0, D_0, mc2)


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/libfk_oracle.so`` (OpenMP if the
    host compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _LIB, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int), ("axis", ctypes.POINTER(ctypes.c_double) * 3)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        gp = ctypes.POINTER(_Grid)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.fko_march.argtypes = [gp, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  dp, dp, ctypes.c_int, ctypes.c_int]
        lib.fko_step_nodes.argtypes = [gp, ctypes.c_int, dp, ctypes.c_int, dp, dp,
                                       ctypes.c_double, ctypes.c_int, dp,
                                       ctypes.c_int64, i64p, dp, ctypes.c_int,
                                       ctypes.c_int]
        lib.fko_interp.argtypes = [gp, dp, ctypes.c_int64, dp, dp]
        lib.fko_slopes.argtypes = [gp, dp, dp]
        lib.fko_slopes.restype = None
        lib.fko_coefficients.argtypes = [ctypes.c_int, dp, ctypes.c_int,
                                         ctypes.c_double, dp, dp, dp]
        lib.fko_coefficients.restype = None
        lib.fko_quench_params.argtypes = [dp, ctypes.c_double, dp]
        lib.fko_quench_params.restype = None
        lib.fko_adjoint.argtypes = [gp, ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_double,
                                    ctypes.c_int, dp, dp, dp, dp]
        _lib = lib
    return _lib


def has_openmp() -> bool:
    return bool(_load().fko_has_openmp())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass(frozen=True)
class Grid:
    """Uniform Cartesian mesh S of Sec. 3.1.2: ``n[m]`` nodes on
    ``[lo[m], hi[m]]`` per axis; fields are stored x fastest.  Bit m of
    ``periodic`` makes axis m periodic: its last node is its first (the
    period is n[m] - 1 nodes) and nothing exits through it.  ``axes[m]``,
    if given, holds the increasing node coordinates of axis m (a
    non-uniform mesh; first = lo[m], last = hi[m])."""
    n: tuple
    lo: tuple
    hi: tuple
    periodic: int = 0
    axes: tuple | None = None

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def size(self) -> int:
        return int(np.prod(self.n))

    @property
    def shape(self) -> tuple:
        """numpy shape of a field (slowest axis first)."""
        return tuple(reversed(self.n))

    def h(self, m: int) -> float:
        return (self.hi[m] - self.lo[m]) / (self.n[m] - 1)

    def axis(self, m: int) -> np.ndarray:
        if self.axes is not None and self.axes[m] is not None:
            return np.asarray(self.axes[m], dtype=np.float64)
        return self.lo[m] + np.arange(self.n[m]) * self.h(m)

    def _c(self) -> _Grid:
        keep = []
        g = _Grid()
        g.dim = self.dim
        for m in range(self.dim):
            g.n[m] = int(self.n[m])
            g.lo[m] = float(self.lo[m])
            g.hi[m] = float(self.hi[m])
            if self.axes is not None and self.axes[m] is not None:
                a = np.ascontiguousarray(self.axes[m], dtype=np.float64)
                if a.size != self.n[m]:
                    raise ValueError("axes[m] must hold n[m] coordinates")
                keep.append(a)
                g.axis[m] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        g.periodic = int(self.periodic)
        g._keep = keep  # the coordinate arrays live as long as the struct
        return g


def _params(p: Sequence[float]) -> np.ndarray:
    out = np.zeros(16, dtype=np.float64)
    out[: len(p)] = p
    return out


# ----------------------------------------------------------- quadrature --

def gauss_hermite(q: int):
    """Golub-Welsch: the nodes are the eigenvalues of the symmetric
    tridiagonal Jacobi matrix of the polynomials orthonormal for
    pi^{-1/2} exp(-xi^2) (zero diagonal, off-diagonal sqrt(k/2)); the weight
    of each node is the squared first component of its unit eigenvector
    (the measure has total mass 1, Eq. (expec)).  Returns (a, w) sorted by a.
    """
    if q < 1:
        raise ValueError("q must be >= 1")
    k = np.arange(1, q, dtype=np.float64)
    jac = np.diag(np.sqrt(k / 2.0), 1) + np.diag(np.sqrt(k / 2.0), -1)
    vals, vecs = np.linalg.eigh(jac)
    w = vecs[0, :] ** 2
    order = np.argsort(vals)
    return vals[order].copy(), w[order].copy()


# ------------------------------------------------------------- fields ----

def terminal_indicator(grid: Grid, family: int = CONST_DRIFT) -> np.ndarray:
    """chi of Sec. 3.2: 0 at interior nodes, 1 at boundary nodes (the faces
    of the non-periodic axes).  The runaway model counts only p = p_max
    (the upper face of axis 0): chi is 1 there and 0 elsewhere."""
    chi = np.zeros(grid.shape, dtype=np.float64)
    if family in (RUNAWAY, RUNAWAY_QUENCH):
        chi[..., -1] = 1.0
        return chi
    for ax in range(chi.ndim):
        if (grid.periodic >> (chi.ndim - 1 - ax)) & 1:
            continue
        sl = [slice(None)] * chi.ndim
        sl[ax] = 0
        chi[tuple(sl)] = 1.0
        sl[ax] = -1
        chi[tuple(sl)] = 1.0
    return chi


def coefficients(family: int, params, dim: int, t: float, x) -> tuple:
    lib = _load()
    p = _params(params)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    b = np.zeros(dim)
    s = np.zeros(dim * dim)
    lib.fko_coefficients(family, _dp(p), dim, float(t), _dp(xx), _dp(b), _dp(s))
    return b, s.reshape(dim, dim)


def quench_params(params, t: float) -> np.ndarray:
    """The static runaway parameters (E, tau, Z, delta, nu_ee, v_T, r_D, W,
    Delta_p, V_0, D_0) of the thermal-quench model at time t."""
    lib = _load()
    out = np.zeros(11)
    lib.fko_quench_params(_dp(_params(params)), float(t), _dp(out))
    return out


def slopes(grid: Grid, u: np.ndarray) -> np.ndarray:
    """PCHIP nodal slopes (Eq. (e300)) of u along each axis; returns an array
    of shape (dim,) + grid.shape."""
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.zeros(grid.dim * grid.size)
    lib.fko_slopes(ctypes.byref(grid._c()), _dp(uu), _dp(out))
    return out.reshape((grid.dim,) + grid.shape)


def interp(grid: Grid, u: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """The interpolant of Eq. (Lag11) at points (npts, dim) inside the box."""
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    pp = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, grid.dim)
    out = np.zeros(pp.shape[0])
    rc = lib.fko_interp(ctypes.byref(grid._c()), _dp(uu), pp.shape[0], _dp(pp), _dp(out))
    if rc:
        raise ValueError(f"fko_interp failed ({rc})")
    return out


def march(grid: Grid, family: int, params, q: int, dt: float, n_from: int,
          n_to: int, u_in: np.ndarray | None = None, nthreads: int = 1,
          boundary_rule: bool = True) -> np.ndarray:
    """Scheme 1 from u^{n_from} to u^{n_to}.  ``u_in=None`` means chi."""
    lib = _load()
    a, w = gauss_hermite(q)
    if u_in is None:
        u_in = terminal_indicator(grid, family)
    uu = np.ascontiguousarray(u_in, dtype=np.float64).reshape(-1)
    if uu.size != grid.size:
        raise ValueError("u_in has the wrong size")
    out = np.zeros(grid.size)
    p = _params(params)
    rc = lib.fko_march(ctypes.byref(grid._c()), family, _dp(p), q, _dp(a), _dp(w),
                       float(dt), int(n_from), int(n_to), _dp(uu), _dp(out),
                       int(nthreads), int(bool(boundary_rule)))
    if rc:
        raise ValueError(f"fko_march failed ({rc})")
    return out.reshape(grid.shape)


def step_nodes(grid: Grid, family: int, params, q: int, dt: float, n: int,
               u_next: np.ndarray, nodes: np.ndarray, nthreads: int = 1,
               boundary_rule: bool = True) -> np.ndarray:
    """u^n at the listed flat node indices, from the full field u^{n+1}."""
    lib = _load()
    a, w = gauss_hermite(q)
    uu = np.ascontiguousarray(u_next, dtype=np.float64).reshape(-1)
    nn = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros(nn.size)
    p = _params(params)
    rc = lib.fko_step_nodes(ctypes.byref(grid._c()), family, _dp(p), q, _dp(a), _dp(w),
                            float(dt), int(n), _dp(uu), nn.size,
                            nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _dp(out), int(nthreads), int(bool(boundary_rule)))
    if rc:
        raise ValueError(f"fko_step_nodes failed ({rc})")
    return out


def adjoint(grid: Grid, family: int, params, q: int, dt: float, n_steps: int,
            cot_u0: np.ndarray, u_terminal: np.ndarray | None = None):
    """Reverse-mode derivative of L = <cot_u0, u^0> over the whole march:
    returns (dL/dp[0..3], dL/du^N).  Keeps every u^n (small grids only)."""
    lib = _load()
    a, w = gauss_hermite(q)
    if u_terminal is None:
        u_terminal = terminal_indicator(grid)
    ut = np.ascontiguousarray(u_terminal, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(cot_u0, dtype=np.float64).reshape(-1)
    dth = np.zeros(4)
    dut = np.zeros(grid.size)
    p = _params(params)
    rc = lib.fko_adjoint(ctypes.byref(grid._c()), family, _dp(p), q, _dp(a), _dp(w), float(dt),
                         int(n_steps), _dp(ut), _dp(g), _dp(dth), _dp(dut))
    if rc:
        raise ValueError(f"fko_adjoint failed ({rc})")
    return dth, dut.reshape(grid.shape)


# ------------------------------------------------------- closed forms ----

def _norm_cdf(x):
    from scipy.special import ndtr
    return ndtr(x)


def exit_prob_1d_image(x, T: float, a: float, b: float, mu: float = 0.0,
                       sigma: float = 1.0, terms: int = 60):
    """P(tau <= T | X_0 = x) for dX = mu dt + sigma dW on (a, b), exit
    monitored continuously.  Method of images for the killed Brownian motion
    combined with the Girsanov factor exp(mu (y - s) - mu^2 T / 2): each
    image at centre c contributes exp(mu (c - s)) [Phi((L - c - mu T)/sqrt T)
    - Phi((-c - mu T)/sqrt T)] with sign +1 for c = s + 2 m L and -1 for
    c = -s + 2 m L (s = x - a, L = b - a), after scaling by sigma."""
    x = np.asarray(x, dtype=np.float64)
    if T <= 0:
        return np.where((x > a) & (x < b), 0.0, 1.0)
    s = (x - a) / sigma
    L = (b - a) / sigma
    m_ = mu / sigma
    rt = math.sqrt(T)
    surv = np.zeros_like(s)
    for m in range(-terms, terms + 1):
        for c, sign in ((s + 2 * m * L, 1.0), (-s + 2 * m * L, -1.0)):
            term = np.exp(m_ * (c - s)) * (_norm_cdf((L - c - m_ * T) / rt)
                                           - _norm_cdf((-c - m_ * T) / rt))
            surv = surv + sign * term
    return 1.0 - surv


def exit_prob_1d_eigen(x, T: float, a: float, b: float, mu: float = 0.0,
                       sigma: float = 1.0, terms: int = 4000):
    """The same probability from the sine eigen-expansion of the killed
    driftless motion and the Girsanov factor:
    S = exp(-mu s - mu^2 T/2) sum_n (2/L) sin(k_n s) exp(-k_n^2 T/2)
        * k_n (1 - (-1)^n exp(mu L)) / (mu^2 + k_n^2),  k_n = n pi / L."""
    x = np.asarray(x, dtype=np.float64)
    s = (x - a) / sigma
    L = (b - a) / sigma
    m_ = mu / sigma
    n = np.arange(1, terms + 1, dtype=np.float64)
    k = n * math.pi / L
    coef = (2.0 / L) * np.exp(-k * k * T / 2.0) * k * (1.0 - (-1.0) ** n * math.exp(m_ * L)) / (m_ * m_ + k * k)
    surv = np.exp(-m_ * s - m_ * m_ * T / 2.0) * (np.sin(np.multiply.outer(s, k)) @ coef)
    return 1.0 - surv


def exit_prob_1d_paper_e45(x, T: float, L: float, terms: int = 4000):
    """Eq. (e45) for X = X_0 + W_t on [0, L], read with odd n only: as printed
    the series runs over every n >= 1, which does not give P = 0 inside the
    interval at T = 0; the sine series of the indicator keeps only odd n."""
    x = np.asarray(x, dtype=np.float64)
    n = np.arange(1, 2 * terms, 2, dtype=np.float64)
    coef = 4.0 / (n * math.pi) * np.exp(-0.5 * (n * math.pi / L) ** 2 * T)
    return 1.0 - np.sin(np.multiply.outer(x, n * math.pi / L)) @ coef


# --------------------------------------------------------- Monte Carlo ---

def _drift_numpy(family: int, params, t: float, x: np.ndarray) -> tuple:
    """b(t, x) for an array of points x (npts, dim) and the scalar sigma,
    the same families as ``fko_coefficients``, written with numpy."""
    if family == CONST_DRIFT:
        d = x.shape[1]
        return np.broadcast_to(np.asarray(params[:d], dtype=np.float64), x.shape), float(params[3])
    if family == PAPER_CELLULAR:
        Pe, nn, eps, omega = params[:4]
        f = math.cos(omega * t)
        X, Y = x[:, 0], x[:, 1]
        bx = -Pe * math.pi * np.cos(math.pi * Y) * (np.sin(nn * X) + eps * f * np.cos(nn * X))
        by = Pe * nn * np.sin(math.pi * Y) * (np.cos(nn * X) - eps * f * np.sin(nn * X))
        return np.stack([bx, by], axis=1), 1.0
    A, eps, omega, D = params[:4]
    f = math.sin(omega * t)
    X, Y = x[:, 0], x[:, 1]
    bx = -math.pi * np.cos(math.pi * Y) * (A * np.sin(math.pi * X) + eps * f * np.sin(2 * math.pi * X))
    by = math.pi * np.sin(math.pi * Y) * (A * np.cos(math.pi * X) + 2 * eps * f * np.cos(2 * math.pi * X))
    return np.stack([bx, by], axis=1), math.sqrt(2.0 * D)


def mc_exit_prob(family: int, params, lo, hi, x0, dt: float, n_steps: int,
                 paths: int, seed: int, chunk: int = 250_000,
                 bridge: bool = False, periodic: int = 0) -> float:
    """Euler-Maruyama (Eq. (ref-X)) from t_0 = 0 over n_steps steps; returns
    the fraction of paths that left the open box by t_N.

    bridge=False checks the exit only at the t_{n+1}.  bridge=True follows
    the footnote to Eq. (e24), where the exit time is that of the
    continuous-time Euler path x + b(t_n,x)(s - t_n) + sigma (W_s - W_{t_n}):
    a path that is inside at both ends of a step is also killed with the
    probability that the Brownian bridge between them crossed a face,
    exp(-2 d_n d_{n+1} / (sigma^2 dt)) per face (d = distance to that
    face), taken as independent across faces.  Bit m of periodic wraps
    axis m onto [lo, hi) instead (no exit through it)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = lo.size
    per = np.array([(periodic >> k) & 1 == 1 for k in range(d)])
    exited = 0
    done = 0
    while done < paths:
        m = min(chunk, paths - done)
        x = np.tile(np.asarray(x0, dtype=np.float64), (m, 1))
        alive = np.ones(m, dtype=bool)
        for n in range(n_steps):
            b, s = _drift_numpy(family, params, n * dt, x)
            xn = x + b * dt + s * math.sqrt(dt) * rng.standard_normal((m, d))
            if per.any():
                xn[:, per] = lo[per] + np.mod(xn[:, per] - lo[per], (hi - lo)[per])
            out = np.any(((xn <= lo) | (xn >= hi)) & ~per, axis=1)
            if bridge and s > 0:
                var = s * s * dt
                stay = np.ones(m)
                for k in range(d):
                    if per[k]:
                        continue
                    dl0, dl1 = x[:, k] - lo[k], xn[:, k] - lo[k]
                    du0, du1 = hi[k] - x[:, k], hi[k] - xn[:, k]
                    stay *= 1.0 - np.exp(-2.0 * np.clip(dl0 * dl1, 0, None) / var)
                    stay *= 1.0 - np.exp(-2.0 * np.clip(du0 * du1, 0, None) / var)
                out |= rng.uniform(size=m) >= stay
            alive &= ~out
            x = xn
        exited += int(m - alive.sum())
        done += m
    return exited / paths
