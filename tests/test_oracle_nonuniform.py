"""Pins for the oracle on non-uniform axes (the mesh of Sec. 3.1.2 need not
be uniform along any direction; Sec. 4.3 uses graded meshes).  Eq. (e300)
is applied as printed: divided differences over the actual spacings and
their plain harmonic mean; the Hermite cell formula takes each cell's own
width.

* Coordinates given explicitly but uniform reproduce the uniform march.
* Affine data on strongly graded axes: the slopes are exact, the
  interpolant reproduces the data, and one step of constant drift maps it to
  the same affine function shifted by b dt (Gauss-Hermite is exact on
  affine integrands): exact to rounding at every node whose points stay in
  the box.
* 1D drifted Brownian motion on a mesh graded towards both faces against
  discretely monitored Monte Carlo, to the tolerance the uniform mesh with
  twice the nodes meets.
* d = 3: explicit uniform coordinates reproduce the uniform march, for
  constant drift and for the runaway-electron model (its coefficients then
  come from the given coordinates and act in physical lengths); affine data
  on three graded axes is reproduced by the tricubic interpolant and shifted
  by b dt by one step.
"""
import math

import numpy as np

import fk_inputs

PATHS = 1_000_000


_graded = fk_inputs.graded_axis


def test_explicit_uniform_axes_reproduce_uniform(oracle):
    n = (45, 29)
    g = oracle.Grid(n, (0.0, 0.0), (2.0, 1.0))
    ga = oracle.Grid(n, (0.0, 0.0), (2.0, 1.0), axes=(g.axis(0), g.axis(1)))
    p = [1.0, 0.2, 2 * math.pi, 0.01]
    u0 = fk_inputs.random_field((29, 45), seed=3)
    a = oracle.march(g, oracle.CELLULAR_FLOW, p, 4, 1e-3, 10, 0, u0)
    b = oracle.march(ga, oracle.CELLULAR_FLOW, p, 4, 1e-3, 10, 0, u0)
    assert np.abs(a - b).max() <= 1e-14


def test_affine_data_on_graded_axes(oracle):
    ax = _graded(-4.0, 4.0, 61, 0.9)
    ay = _graded(-3.0, 3.0, 47, 0.7)
    assert (np.diff(ax).max() / np.diff(ax).min()) > 10
    g = oracle.Grid((61, 47), (-4.0, -3.0), (4.0, 3.0), axes=(ax, ay))
    X, Y = np.meshgrid(ax, ay)
    u = 0.3 + 0.05 * X - 0.07 * Y
    b, s, dt = (0.6, -0.4), 0.5, 0.01
    got = oracle.march(g, oracle.CONST_DRIFT, [b[0], b[1], 0.0, s], 6, dt, 1, 0, u,
                       boundary_rule=False)
    want = 0.3 + 0.05 * (X + b[0] * dt) - 0.07 * (Y + b[1] * dt)
    a, _ = oracle.gauss_hermite(6)
    reach = max(abs(b[0]), abs(b[1])) * dt + s * math.sqrt(2 * dt) * abs(a).max()
    inside = (np.abs(X) < 4.0 - reach - 1e-9) & (np.abs(Y) < 3.0 - reach - 1e-9)
    assert inside.sum() > 1500
    assert np.abs(got - want)[inside].max() <= 1e-13
    # the interpolant itself, at random points
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(-4, 4, 500), rng.uniform(-3, 3, 500)], axis=1)
    vals = oracle.interp(g, u, pts)
    assert np.abs(vals - (0.3 + 0.05 * pts[:, 0] - 0.07 * pts[:, 1])).max() <= 1e-13


def test_graded_1d_monte_carlo(oracle):
    dt, N = 0.005, 200
    p = [0.5, 0.0, 0.0, 1.0]
    ax = _graded(-1.0, 1.0, 401, 0.6)
    g = oracle.Grid((401,), (-1.0,), (1.0,), axes=(ax,))
    u = oracle.march(g, oracle.CONST_DRIFT, p, 8, dt, N, 0)
    for j, seed in ((200, 21), (300, 22), (60, 23), (380, 24)):
        x0 = float(ax[j])
        mc = oracle.mc_exit_prob(oracle.CONST_DRIFT, p, [-1.0], [1.0], [x0], dt, N, PATHS,
                                 seed=seed)
        tol = 4 * math.sqrt(mc * (1 - mc) / PATHS) + 2.5e-3
        assert abs(u[j] - mc) < tol, (x0, u[j], mc, tol)


def test_explicit_uniform_axes_reproduce_uniform_3d(oracle):
    runaway = fk_inputs.workload("runaway_97x65x41")["params"]
    cases = (((13, 11, 9), (-1.0,) * 3, (1.0,) * 3, oracle.CONST_DRIFT, [0.3, -0.2, 0.1, 0.4],
              2e-3),
             ((13, 9, 11), (2.0, -1.0, 0.0), (12.0, 1.0, 1.0), oracle.RUNAWAY, list(runaway),
              0.05))
    for n, lo, hi, fam, p, dt in cases:
        g = oracle.Grid(n, lo, hi)
        ga = oracle.Grid(n, lo, hi, axes=tuple(g.axis(m) for m in range(3)))
        u0 = fk_inputs.random_field(tuple(reversed(n)), seed=4, boundary_one=False) \
            if fam == oracle.CONST_DRIFT else None
        a = oracle.march(g, fam, p, 4, dt, 8, 0, u0)
        b = oracle.march(ga, fam, p, 4, dt, 8, 0, u0)
        assert np.abs(a).max() > 0.05
        assert np.abs(a - b).max() <= 1e-13, fam


def test_affine_data_on_graded_axes_3d(oracle):
    axs = (_graded(-2.0, 2.0, 25, 0.9), _graded(-1.5, 1.5, 21, 0.85), _graded(-1.0, 1.0, 17, 0.8))
    assert min(np.diff(a).max() / np.diff(a).min() for a in axs) > 4
    g = oracle.Grid((25, 21, 17), (-2.0, -1.5, -1.0), (2.0, 1.5, 1.0), axes=axs)
    Z, Y, X = np.meshgrid(axs[2], axs[1], axs[0], indexing="ij")
    c = (0.3, 0.05, -0.07, 0.04)
    u = c[0] + c[1] * X + c[2] * Y + c[3] * Z
    b, s, dt = (0.6, -0.4, 0.3), 0.3, 0.01
    got = oracle.march(g, oracle.CONST_DRIFT, [b[0], b[1], b[2], s], 4, dt, 1, 0, u,
                       boundary_rule=False)
    want = c[0] + c[1] * (X + b[0] * dt) + c[2] * (Y + b[1] * dt) + c[3] * (Z + b[2] * dt)
    a, _ = oracle.gauss_hermite(4)
    reach = max(abs(v) for v in b) * dt + s * math.sqrt(2 * dt) * abs(a).max()
    inside = ((np.abs(X) < 2.0 - reach - 1e-9) & (np.abs(Y) < 1.5 - reach - 1e-9)
              & (np.abs(Z) < 1.0 - reach - 1e-9))
    assert inside.sum() > 3000
    assert np.abs(got - want)[inside].max() <= 1e-13
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(-2, 2, 400), rng.uniform(-1.5, 1.5, 400),
                    rng.uniform(-1, 1, 400)], axis=1)
    vals = oracle.interp(g, u, pts)
    ref = c[0] + c[1] * pts[:, 0] + c[2] * pts[:, 1] + c[3] * pts[:, 2]
    assert np.abs(vals - ref).max() <= 1e-13
