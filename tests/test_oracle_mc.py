"""Pins for the oracle's march against Euler-Maruyama Monte Carlo.

When shifted points can leave the box (Assumption 1, Eq. (e301), violated),
the scheme is the Markov chain that checks the exit only at the t_n (the
footnote to Eq. (e24)), evaluated with Gauss-Hermite quadrature and the
PCHIP interpolant.  It then differs from the discretely monitored Monte
Carlo estimate only by quadrature and interpolation error; the largest part
sits in the last cell before the boundary, where the discretely monitored
solution jumps to the boundary value 1, so it shrinks with the mesh width.
We check:
* 1D, drift 0.5, sigma 1 on (-1, 1), dt = 5e-3, 200 steps, 801 nodes:
  agreement within 4 standard errors of 10^6 paths plus the measured
  interpolation error at this mesh width (2.5e-3);
* 2D cellular flow (A = 1, eps = 0.2, omega = 2 pi, D = 0.02), dt = 1e-3,
  200 steps: the gap to Monte Carlo shrinks as the mesh is refined from
  33 to 129 rows and is below 0.035 there.
"""
import math

import numpy as np

PATHS_1D = 1_000_000


def test_mc_1d_discrete(oracle):
    dt, N = 0.005, 200
    p = [0.5, 0.0, 0.0, 1.0]
    g = oracle.Grid((801,), (-1.0,), (1.0,))
    u = oracle.march(g, oracle.CONST_DRIFT, p, 8, dt, N, 0)
    for x0, j, seed in ((0.0, 400, 11), (0.5, 600, 12), (-0.7, 120, 13)):
        assert abs(g.axis(0)[j] - x0) < 1e-12
        mc = oracle.mc_exit_prob(oracle.CONST_DRIFT, p, [-1.0], [1.0], [x0], dt, N,
                                 PATHS_1D, seed=seed)
        tol = 4 * math.sqrt(mc * (1 - mc) / PATHS_1D) + 2.5e-3
        assert abs(u[j] - mc) < tol, (x0, u[j], mc, tol)


def test_mc_2d_cellular_refinement(oracle):
    dt, N = 1e-3, 200
    p = [1.0, 0.2, 2 * math.pi, 0.02]
    x0 = (0.25, 0.0625)
    paths = 250_000
    mc = oracle.mc_exit_prob(oracle.CELLULAR_FLOW, p, [0, 0], [2, 1], list(x0), dt, N, paths,
                             seed=5)
    gaps = []
    for ny in (33, 129):
        nx = 2 * (ny - 1) + 1
        g = oracle.Grid((nx, ny), (0.0, 0.0), (2.0, 1.0))
        u = oracle.march(g, oracle.CELLULAR_FLOW, p, 6, dt, N, 0, nthreads=8)
        i, k = int(round(x0[0] / g.h(0))), int(round(x0[1] / g.h(1)))
        gaps.append(abs(u[k, i] - mc))
    noise = 4 * math.sqrt(mc * (1 - mc) / paths)
    assert gaps[1] < 0.5 * gaps[0]
    assert gaps[1] < 0.035 + noise, gaps
