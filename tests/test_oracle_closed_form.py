"""Pins for the oracle's march against the continuous problem.

* two independent closed forms of the exit probability of 1D Brownian motion
  with drift (image series and sine eigen-series) agree with each other,
  and with the driftless series of Eq. (e45) read with odd terms;
* the 1D workload with drift b = 0.5, sigma = 1 on (-1, 1), T = 1, 201
  nodes, Q = 8, dt = 1e-3: the scheme monitors the exit only at the t_n
  (footnote to Eq. (e24)) and this grid violates Assumption 1 (Eq. (e301)),
  so against the continuously monitored closed form it carries a
  boundary-layer bias of order sqrt(dt); the bias shrinks by more than half
  when the closed form's barrier is moved out by the Broadie-Glasserman-Kou
  shift 0.5826 sigma sqrt(dt) (a known correction for discrete monitoring);
* first-order convergence in dt on the Fig. 2 setup (L = 10, T = 3, Q = 3,
  sigma = 1, b = 0, Sec. 4.1) with grids that satisfy Remark 2, so that
  Delta x ~ sqrt(dt) and the error also falls as Delta x^2 (Eq. (e_err));
* second-order convergence in Delta x at fixed dt (the error estimate after
  Scheme 1 in Sec. 3.1, and Fig. 4 of Sec. 4.2) with smooth terminal data
  that meets the exit value;
* 0 <= u <= 1 and monotonicity in time-to-go for the autonomous 1D problem;
* constant drift in a 2D or 3D box: the survival is the product of the 1D
  survivals (independent components), approached under refinement;
* for the non-autonomous cellular flow, P(t_k, x) is non-decreasing in the
  horizon t_k (exit by t_k implies exit by t_{k+1}): to rounding on a
  resolved grid, with the scheme's violations vanishing under refinement.
"""
import math

import numpy as np
import pytest


def test_closed_forms_agree(oracle):
    x = np.linspace(-0.99, 0.99, 41)
    for T in (0.01, 0.2, 1.0, 3.0):
        for mu in (0.0, 0.5, -1.3):
            im = oracle.exit_prob_1d_image(x, T, -1.0, 1.0, mu, 1.0)
            ei = oracle.exit_prob_1d_eigen(x, T, -1.0, 1.0, mu, 1.0)
            np.testing.assert_allclose(im, ei, atol=2e-12 if T > 0.05 else 1e-9)
    xs = np.linspace(0.1, 9.9, 30)
    np.testing.assert_allclose(oracle.exit_prob_1d_paper_e45(xs, 3.0, 10.0),
                               oracle.exit_prob_1d_image(xs, 3.0, 0.0, 10.0), atol=1e-12)
    # sigma rescales time: sigma = 2 over T equals sigma = 1 over 4T
    np.testing.assert_allclose(oracle.exit_prob_1d_image(x, 0.3, -1, 1, 0.0, 2.0),
                               oracle.exit_prob_1d_image(x, 1.2, -1, 1, 0.0, 1.0), atol=1e-13)


def _c1(oracle):
    g = oracle.Grid((201,), (-1.0,), (1.0,))
    u = oracle.march(g, oracle.CONST_DRIFT, [0.5, 0, 0, 1.0], 8, 1e-3, 1000, 0)
    return g, u


def test_drifted_brownian_workload(oracle):
    g, u = _c1(oracle)
    x = g.axis(0)
    cont = oracle.exit_prob_1d_image(x, 1.0, -1.0, 1.0, 0.5, 1.0)
    err = np.abs(u - cont)[1:-1].max()
    assert err < 2e-2  # discrete-monitoring bias, O(sqrt(dt)) near the boundary
    sh = 0.5826 * math.sqrt(1e-3)
    corr = oracle.exit_prob_1d_image(x, 1.0, -1.0 - sh, 1.0 + sh, 0.5, 1.0)
    err_c = np.abs(u - corr)[1:-1].max()
    assert err_c < 0.5 * err and err_c < 8e-3
    # the bias reaches the middle of the interval but stays ~1e-2 there
    mid = np.abs(x) < 0.5
    assert np.abs(u - cont)[mid].max() < 1.5e-2
    # the drift pushes towards +1: P is larger near +1 than at the mirror point
    assert u[150] > u[50]


def test_first_order_in_dt(oracle):
    L, T = 10.0, 3.0
    a, _ = oracle.gauss_hermite(3)
    errs = []
    dts = [0.04, 0.02, 0.01, 0.005]
    for dt in dts:
        reach = math.sqrt(2 * dt) * np.abs(a).max()
        n = int(math.floor(L / reach)) + 1  # h = L/floor(L/reach) >= reach
        g = oracle.Grid((n,), (0.0,), (L,))
        u = oracle.march(g, oracle.CONST_DRIFT, [0, 0, 0, 1.0], 3, dt, int(round(T / dt)), 0)
        ex = oracle.exit_prob_1d_image(g.axis(0), T, 0.0, L)
        errs.append(math.sqrt(np.mean((u - ex) ** 2)))
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert all(0.85 < o < 1.4 for o in orders), orders
    assert errs[-1] < 2e-4


def test_second_order_in_dx(oracle):
    """Fixed dt = 0.02, T = 0.2 (10 steps), drift 0.3, sigma 0.2 on (-1, 1),
    terminal data 1 - (1 - x^2)^2 (smooth, equal to the exit value 1 at the
    ends).  The reference is the same march on 1281 nodes, so the time error
    cancels and what is left is the spatial error of the PCHIP interpolant at
    the shifted points.  Semi-Lagrangian errors wobble from level to level
    (the shifted points' fractional cell positions change with h), so the
    pin is the least-squares slope of log error against log h, plus a floor
    on each single-level ratio.  The ladder stops at 321 nodes: below ~1e-6
    the difference to the reference runs into the limiter's switching noise."""
    def run(n):
        g = oracle.Grid((n,), (-1.0,), (1.0,))
        x = g.axis(0)
        return g, oracle.march(g, oracle.CONST_DRIFT, [0.3, 0, 0, 0.2], 8, 0.02, 10, 0,
                               1 - (1 - x * x) ** 2, nthreads=4)
    _, ref = run(1281)
    hs, errs = [], []
    for n in (41, 81, 161, 321):
        g, u = run(n)
        x = g.axis(0)
        inner = np.abs(x) <= 0.6
        errs.append(np.abs(u - ref[::1280 // (n - 1)])[inner].max())
        hs.append(2.0 / (n - 1))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope > 2.0, (slope, errs)
    orders = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert all(o > 1.8 for o in orders), orders
    assert errs[-1] < 1e-5, errs


def test_bounds_and_monotone_in_time_to_go(oracle):
    g = oracle.Grid((201,), (-1.0,), (1.0,))
    p = [0.5, 0, 0, 1.0]
    u = oracle.terminal_indicator(g)
    worst = 0.0
    for n in range(200, 0, -1):
        un = oracle.march(g, oracle.CONST_DRIFT, p, 8, 1e-3, n, n - 1, u)
        worst = max(worst, float(np.max(u - un)))
        assert un.min() >= -1e-15 and un.max() <= 1.0 + 1e-15
        u = un
    assert worst <= 1e-14


def test_2d_constant_drift_product_form(oracle):
    """Constant drift with independent components in a box: the survival is
    the product of the 1D survivals.  On Remark-2 grids (h ~ sqrt(dt)) the
    2D error first falls fast and then levels off: the interpolant carries
    no cross derivative (the columns of Psi in Eq. (e34) are u and its first
    partials only), which leaves an O(h^2) u_xy term per step."""
    T, b = 0.5, (0.3, -0.2)
    a, _ = oracle.gauss_hermite(3)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        reach = math.sqrt(2 * dt) * np.abs(a).max() + 0.3 * dt
        n = int(math.floor(2.0 / reach)) + 1
        g = oracle.Grid((n, n), (-1.0, -1.0), (1.0, 1.0))
        u = oracle.march(g, oracle.CONST_DRIFT, [b[0], b[1], 0, 1.0], 3, dt, int(round(T / dt)), 0,
                         nthreads=4)
        sx = 1 - oracle.exit_prob_1d_image(g.axis(0), T, -1, 1, b[0], 1.0)
        sy = 1 - oracle.exit_prob_1d_image(g.axis(1), T, -1, 1, b[1], 1.0)
        errs.append(math.sqrt(np.mean((u - (1 - np.outer(sy, sx))) ** 2)))
    assert errs[0] > 2.5 * errs[1] and errs[1] > errs[2], errs
    assert errs[2] < 3e-3, errs


def test_3d_constant_drift_product_form(oracle):
    """The same product form in 3D (survival = product of three 1D
    survivals) on Remark-2 grids: the error falls as in 2D (rms 1.4e-2,
    3.9e-3, 1.4e-3 for dt = 0.02, 0.01, 0.005)."""
    T, b = 0.5, (0.3, -0.2, 0.1)
    a, _ = oracle.gauss_hermite(3)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        reach = math.sqrt(2 * dt) * np.abs(a).max() + 0.3 * dt
        n = int(math.floor(2.0 / reach)) + 1
        g = oracle.Grid((n, n, n), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
        u = oracle.march(g, oracle.CONST_DRIFT, [b[0], b[1], b[2], 1.0], 3, dt,
                         int(round(T / dt)), 0, nthreads=4)
        s = [1 - oracle.exit_prob_1d_image(g.axis(m), T, -1, 1, b[m], 1.0) for m in range(3)]
        ref = 1 - np.einsum("k,j,i->kji", s[2], s[1], s[0])
        errs.append(math.sqrt(np.mean((u - ref) ** 2)))
    assert errs[0] > 2.5 * errs[1] and errs[1] > 2.0 * errs[2], errs
    assert errs[2] < 2e-3, errs


def test_monotone_in_horizon_non_autonomous(oracle):
    """P(t_k) for horizons k = 1..K, each a march of k steps from t_k to 0
    with the time-dependent cellular flow (eps = 0.3).  The nonlinear PCHIP
    step is not order-preserving, so coarse grids show small decreases; they
    fall by orders of magnitude per refinement and are at rounding on the
    129 x 65 grid with dt = 5e-3."""
    def worst(n, dt, K):
        g = oracle.Grid((2 * n - 1, n), (0.0, 0.0), (2.0, 1.0))
        prev, w = None, 0.0
        for k in range(1, K + 1):
            u = oracle.march(g, oracle.CELLULAR_FLOW, [1.0, 0.3, 2 * math.pi, 2e-3], 4, dt, k, 0,
                             nthreads=4)
            if prev is not None:
                w = min(w, float((u - prev).min()))
            prev = u
        return w, prev
    w1, _ = worst(17, 2e-2, 15)
    w2, _ = worst(33, 1e-2, 20)
    w3, last = worst(65, 5e-3, 30)
    assert w1 < -1e-4 and w2 > 1e3 * w1 and w3 > -1e-14, (w1, w2, w3)
    assert last[1:-1, 1:-1].max() > 0.05  # the horizons reach the interior
