"""Pins for the oracle's periodic axis and the paper's own 2D example
(Sec. 4.2: dx = Pe v dt + dW on [-pi, pi] x [0, 1], periodic in x_1,
exit through x_2 = 0 and 1).

* A field and coefficients that do not depend on x, periodic in x: the 2D
  march equals the 1D march along y (no point exits through the x faces).
* Periodic in x equals the non-periodic march on three tiled periods, whose
  middle period is far from the x faces: an independent check of the wrap of
  the shifted points and of the slopes across the seam.
* The paper's velocity field: divergence free, stagnation points at the
  roll centres (+-pi/4, 1/2), (+-3 pi/4, 1/2) and the hyperbolic points
  (0, 0), (+-pi/2, 0), (pi, 0) for n = 2, eps = 0, and the mirror symmetry
  x_1 -> -x_1 (v_1 odd, v_2 even) that the march then keeps.
* Monte Carlo of the time-dependent, periodic example: the gap to the
  discretely monitored estimate shrinks under mesh refinement.
"""
import math

import numpy as np

import fk_inputs

PAPER = [10.0, 2.0, 0.15, 2 * math.pi / 10]  # Pe, n, eps, omega


def test_periodic_x_independent_equals_1d(oracle):
    p = [0.7, 0.3, 0.0, 0.8]
    g2 = oracle.Grid((41, 33), (0.0, -1.0), (2.0, 1.0), periodic=1)
    g1 = oracle.Grid((33,), (-1.0,), (1.0,))
    u2 = oracle.march(g2, oracle.CONST_DRIFT, p, 4, 2e-3, 20, 0)
    u1 = oracle.march(g1, oracle.CONST_DRIFT, [0.3, 0.0, 0.0, 0.8], 4, 2e-3, 20, 0)
    assert np.abs(u2 - u1[:, None]).max() <= 1e-13
    assert u1[1:-1].max() > 0.1


def test_periodic_equals_three_tiled_periods(oracle):
    """One period [0, 2) with 40 cells against [-2, 4] with 120 cells and
    the field tiled three times; after 8 steps nothing from the outer x
    faces has reached the middle period."""
    P, ny = 40, 25
    g = oracle.Grid((P + 1, ny), (0.0, 0.0), (2.0, 1.0), periodic=1)
    gw = oracle.Grid((3 * P + 1, ny), (-2.0, 0.0), (4.0, 1.0))
    u0 = fk_inputs.random_field((ny, P + 1), seed=31)
    u0[:, P] = u0[:, 0]
    wide = np.concatenate([u0[:, :P]] * 3 + [u0[:, :1]], axis=1)
    wide[:, 0] = wide[:, -1] = 0.5  # the far x faces hold 1 anyway
    for fam, p in ((oracle.CONST_DRIFT, [0.9, -0.4, 0.0, 0.5]), (oracle.PAPER_CELLULAR, PAPER)):
        gp = g if fam == oracle.CONST_DRIFT else oracle.Grid((P + 1, ny), (-math.pi, 0.0),
                                                              (math.pi, 1.0), periodic=1)
        gwp = gw if fam == oracle.CONST_DRIFT else oracle.Grid(
            (3 * P + 1, ny), (-3 * math.pi, 0.0), (3 * math.pi, 1.0))
        dt = 2e-3 if fam == oracle.CONST_DRIFT else 2e-4
        u = oracle.march(gp, fam, p, 4, dt, 8, 0, u0)
        uw = oracle.march(gwp, fam, p, 4, dt, 8, 0, wide)
        assert np.abs(u - uw[:, P:2 * P + 1]).max() <= 1e-13, fam
        assert np.abs(u - u0).max() > 1e-3


def test_paper_velocity_field(oracle):
    rng = np.random.default_rng(3)
    eps0 = [10.0, 2.0, 0.0, PAPER[3]]

    def b(p, t, x, y):
        return oracle.coefficients(oracle.PAPER_CELLULAR, p, 2, t, [x, y])[0]

    # divergence free (central differences)
    for _ in range(20):
        x, y, t = rng.uniform(-math.pi, math.pi), rng.uniform(0, 1), rng.uniform(0, 10)
        e = 1e-5
        div = ((b(PAPER, t, x + e, y)[0] - b(PAPER, t, x - e, y)[0]) +
               (b(PAPER, t, x, y + e)[1] - b(PAPER, t, x, y - e)[1])) / (2 * e)
        assert abs(div) < 1e-6
    # stagnation points of the unperturbed flow
    for x, y in ((math.pi / 4, 0.5), (-math.pi / 4, 0.5), (3 * math.pi / 4, 0.5),
                 (-3 * math.pi / 4, 0.5), (0.0, 0.0), (math.pi / 2, 0.0), (-math.pi / 2, 0.0),
                 (math.pi, 0.0), (math.pi / 2, 1.0)):
        assert np.abs(b(eps0, 0.0, x, y)).max() < 1e-12, (x, y)
    # elsewhere it moves, and the rolls turn: v_2 changes sign across x_1 = pi/4
    assert abs(b(eps0, 0.0, 0.0, 0.5)[1]) > 10
    assert b(eps0, 0.0, 0.1, 0.5)[1] * b(eps0, 0.0, 1.4, 0.5)[1] < 0
    # mirror x_1 -> -x_1 at eps = 0: v_1 odd, v_2 even; the perturbation breaks it
    for _ in range(10):
        x, y = rng.uniform(-math.pi, math.pi), rng.uniform(0, 1)
        v, m = b(eps0, 0.0, x, y), b(eps0, 0.0, -x, y)
        assert abs(v[0] + m[0]) < 1e-12 and abs(v[1] - m[1]) < 1e-12
    assert oracle.coefficients(oracle.PAPER_CELLULAR, PAPER, 2, 0.0, [0.3, 0.4])[1][0, 0] == 1.0


def test_paper_march_mirror_symmetry(oracle):
    P, ny = 64, 33
    g = oracle.Grid((P + 1, ny), (-math.pi, 0.0), (math.pi, 1.0), periodic=1)
    u = oracle.march(g, oracle.PAPER_CELLULAR, [10.0, 2.0, 0.0, PAPER[3]], 4, 1e-3, 20, 0,
                     nthreads=4)
    mirror = u[:, (P - np.arange(P + 1)) % P]
    assert np.abs(u - mirror).max() <= 1e-13
    assert np.abs(u[:, 0] - u[:, P]).max() == 0.0
    # the perturbed flow is not mirror symmetric
    ue = oracle.march(g, oracle.PAPER_CELLULAR, PAPER, 4, 1e-3, 20, 0, nthreads=4)
    assert np.abs(ue - ue[:, (P - np.arange(P + 1)) % P]).max() > 1e-4


def test_paper_mc_refinement(oracle):
    """Pe = 10, n = 2, eps = 0.15, omega = 2 pi / 10, T = 0.05 (the paper's
    parameters), dt = 5e-4: the march against discretely monitored Monte
    Carlo at a point near a separatrix, on two meshes."""
    dt, N, paths = 5e-4, 100, 200_000
    x0 = (math.pi / 2, 0.125)
    mc = oracle.mc_exit_prob(oracle.PAPER_CELLULAR, PAPER, [-math.pi, 0.0], [math.pi, 1.0],
                             list(x0), dt, N, paths, seed=7, periodic=1)
    gaps = []
    for ny in (33, 129):
        P = 4 * (ny - 1)
        g = oracle.Grid((P + 1, ny), (-math.pi, 0.0), (math.pi, 1.0), periodic=1)
        u = oracle.march(g, oracle.PAPER_CELLULAR, PAPER, 6, dt, N, 0, nthreads=8)
        i = int(round((x0[0] + math.pi) / g.h(0)))
        k = int(round(x0[1] / g.h(1)))
        assert abs(g.axis(0)[i] - x0[0]) < 1e-12 and abs(g.axis(1)[k] - x0[1]) < 1e-12
        gaps.append(abs(u[k, i] - mc))
    noise = 4 * math.sqrt(mc * (1 - mc) / paths)
    print(f"paper example: MC {mc:.4f}, gaps {gaps}")
    assert 0.05 < mc < 0.95
    assert gaps[1] < 0.5 * gaps[0] or gaps[1] < noise
    assert gaps[1] < 0.02 + noise, gaps
