"""Pins for the oracle's interpolant: the PCHIP nodal-slope rule (Eq. (e300)
and its end rule) and the Hermite interpolant of Eq. (Lag11).

* interior slopes and interior cells against scipy's PCHIP, which on a
  uniform grid uses the same harmonic-mean rule (Fritsch-Butland), but a
  different end formula, so only interior cells are compared;
* the end rule read literally from the sentence after Eq. (e300);
* affine data reproduced exactly in 1D, 2D and 3D;
* monotone data gives a monotone interpolant, and each 1D cell stays within
  its end values (shape preservation, Sec. 3.1.2);
* the 2D interpolant against an independent dense sum over the global
  cardinal Hermite functions of each node (the columns of Psi, Eq. (e34)).
"""
import numpy as np
import pytest
from scipy.interpolate import PchipInterpolator


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_interior_slopes_match_scipy(oracle):
    rng = _rng(1)
    g = oracle.Grid((41,), (-1.0,), (3.0,))
    x = g.axis(0)
    for _ in range(5):
        u = np.cumsum(rng.standard_normal(41)) * 0.3
        d = oracle.slopes(g, u)[0]
        ref = PchipInterpolator(x, u).derivative()(x)
        np.testing.assert_allclose(d[1:-1], ref[1:-1], rtol=1e-12, atol=1e-13)


def test_end_slopes_literal_rule(oracle):
    g = oracle.Grid((6,), (0.0,), (5.0,))  # h = 1, deltas are differences
    u = np.array([0.0, 1.0, 3.0, 4.0, 4.5, 7.0])
    d = oracle.slopes(g, u)[0]
    # delta = [1, 2, 1, 0.5, 2.5]
    hm = lambda a, b: 0.0 if a * b <= 0 else 2.0 / (1.0 / a + 1.0 / b)
    assert d[0] == pytest.approx(hm(1.0, 2.0), abs=1e-15)
    assert d[5] == pytest.approx(hm(2.5, 0.5), abs=1e-15)
    assert d[2] == pytest.approx(hm(2.0, 1.0), abs=1e-15)
    # opposite signs and a zero difference both give a zero slope
    u2 = np.array([0.0, 1.0, 0.5, 0.5, 0.7, 0.2])
    d2 = oracle.slopes(g, u2)[0]
    assert d2[1] == 0.0 and d2[2] == 0.0 and d2[3] == 0.0 and d2[4] == 0.0


def test_interior_cells_match_scipy(oracle):
    rng = _rng(2)
    g = oracle.Grid((33,), (0.0,), (2.0,))
    x = g.axis(0)
    u = np.sin(3 * x) + 0.2 * rng.standard_normal(33)
    pts = rng.uniform(x[1], x[-2], size=500)
    got = oracle.interp(g, u, pts[:, None])
    ref = PchipInterpolator(x, u)(pts)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_affine_reproduced(dim, oracle):
    rng = _rng(3 + dim)
    n = (9, 7, 5)[:dim]
    lo = (-1.0, 0.5, 2.0)[:dim]
    hi = (1.0, 2.0, 3.0)[:dim]
    g = oracle.Grid(n, lo, hi)
    c0 = 0.3
    c = rng.standard_normal(dim)
    mesh = np.meshgrid(*[g.axis(m) for m in reversed(range(dim))], indexing="ij")
    coords = list(reversed(mesh))  # coords[m] varies along axis m
    u = c0 + sum(c[m] * coords[m] for m in range(dim))
    pts = np.stack([rng.uniform(lo[m], hi[m], 300) for m in range(dim)], axis=1)
    got = oracle.interp(g, u, pts)
    np.testing.assert_allclose(got, c0 + pts @ c, atol=1e-13)


def test_monotone_and_cell_bounded(oracle):
    rng = _rng(4)
    g = oracle.Grid((25,), (0.0,), (1.0,))
    u = np.sort(rng.uniform(0, 1, 25))
    pts = np.linspace(0, 1, 5001)
    v = oracle.interp(g, u, pts[:, None])
    assert np.all(np.diff(v) >= -1e-15)
    # non-monotone data: every cell stays within its end values
    u = rng.uniform(0, 1, 25)
    v = oracle.interp(g, u, pts[:, None])
    cell = np.minimum((pts / g.h(0)).astype(int), 23)
    lo_ = np.minimum(u[cell], u[cell + 1])
    hi_ = np.maximum(u[cell], u[cell + 1])
    assert np.all(v >= lo_ - 1e-14) and np.all(v <= hi_ + 1e-14)


def _cardinal(xn, h, x):
    """Global cardinal cubic Hermite functions of node xn: value function
    1 - 3 r^2 + 2 r^3 and derivative function (x - xn)(1 - r)^2, r = |x-xn|/h,
    both zero for r >= 1."""
    r = np.abs(x - xn) / h
    inside = r < 1.0
    val = np.where(inside, 1 - 3 * r ** 2 + 2 * r ** 3, 0.0)
    der = np.where(inside, (x - xn) * (1 - r) ** 2, 0.0)
    return val, der


def test_2d_against_dense_cardinal_sum(oracle):
    rng = _rng(5)
    g = oracle.Grid((7, 5), (0.0, -1.0), (3.0, 1.0))
    u = rng.uniform(0, 1, g.shape)  # shape (ny, nx)
    du = oracle.slopes(g, u)  # du[0] = d/dx, du[1] = d/dy
    pts = np.stack([rng.uniform(0, 3, 200), rng.uniform(-1, 1, 200)], axis=1)
    xs, ys = g.axis(0), g.axis(1)
    want = np.zeros(len(pts))
    for k, yk in enumerate(ys):
        vy, dy = _cardinal(yk, g.h(1), pts[:, 1])
        for i, xi in enumerate(xs):
            vx, dx = _cardinal(xi, g.h(0), pts[:, 0])
            want += vx * vy * u[k, i] + dx * vy * du[0][k, i] + vx * dy * du[1][k, i]
    got = oracle.interp(g, u, pts)
    np.testing.assert_allclose(got, want, atol=1e-13)
