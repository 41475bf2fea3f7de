"""Pins for one step of the oracle's Scheme 1 (Sec. 3.1.5).

* the cellular-flow drift is the rotated gradient of its stream function,
  checked by central differences of psi (a sign, factor or argument error
  in the drift fails here);
* affine u maps to affine u shifted by b(t_n, x_j) dt (Gauss-Hermite
  exactness for degree 1 plus affine reproduction of the interpolant),
  including a time-dependent drift, which pins the coefficient time t_n;
* a brute-force dense evaluation of the matrix form u^n = Q Psi^n F^n u^{n+1}
  (Eqs. (e34)-(e36)) with Psi built from global cardinal functions, slopes
  F written independently here, and the exit value 1 for outside queries;
* boundary nodes are held at 1 (Eq. (e3)).
"""
import math

import numpy as np
import pytest

CELL = dict(A=1.0, eps=0.2, omega=2 * math.pi, D=1e-3)


def _psi(x, y, t, A, eps, omega):
    return A * np.sin(np.pi * x) * np.sin(np.pi * y) + eps * np.sin(omega * t) * np.sin(2 * np.pi * x) * np.sin(np.pi * y)


def test_cellular_drift_is_rotated_gradient(oracle):
    rng = np.random.default_rng(0)
    p = [CELL["A"], CELL["eps"], CELL["omega"], CELL["D"]]
    e = 1e-6
    for _ in range(50):
        x, y, t = rng.uniform(0, 2), rng.uniform(0, 1), rng.uniform(0, 3)
        b, s = oracle.coefficients(oracle.CELLULAR_FLOW, p, 2, t, [x, y])
        dpdx = (_psi(x + e, y, t, *p[:3]) - _psi(x - e, y, t, *p[:3])) / (2 * e)
        dpdy = (_psi(x, y + e, t, *p[:3]) - _psi(x, y - e, t, *p[:3])) / (2 * e)
        assert b[0] == pytest.approx(-dpdy, abs=1e-7)
        assert b[1] == pytest.approx(dpdx, abs=1e-7)
        np.testing.assert_allclose(s, math.sqrt(2 * CELL["D"]) * np.eye(2), atol=1e-15)


def _affine_field(g, c0, c):
    mesh = np.meshgrid(*[g.axis(m) for m in reversed(range(g.dim))], indexing="ij")
    coords = list(reversed(mesh))
    return c0 + sum(c[m] * coords[m] for m in range(g.dim)), coords


@pytest.mark.parametrize("case", ["const1d", "const2d", "cell2d", "const3d"])
def test_affine_maps_to_shifted_affine(case, oracle):
    rng = np.random.default_rng(1)
    dt = 2e-3
    if case == "const1d":
        g = oracle.Grid((61,), (-3.0,), (3.0,))
        fam, p = oracle.CONST_DRIFT, [0.7, 0, 0, 0.8]
    elif case == "const2d":
        g = oracle.Grid((31, 21), (-2.0, -1.0), (2.0, 1.0))
        fam, p = oracle.CONST_DRIFT, [-0.4, 0.9, 0, 0.5]
    elif case == "const3d":
        g = oracle.Grid((17, 13, 11), (-2.0, -1.0, 0.0), (2.0, 1.0, 1.0))
        fam, p = oracle.CONST_DRIFT, [0.6, -0.8, 0.3, 0.4]
    else:
        g = oracle.Grid((41, 21), (-1.0, -1.0), (3.0, 2.0))
        fam, p = oracle.CELLULAR_FLOW, [1.3, 0.4, 2 * math.pi, 0.02]
    c = rng.standard_normal(g.dim)
    u, coords = _affine_field(g, 0.25, c)
    n = 37  # t_n = 0.074, sin(omega t_n) != 0
    un = oracle.march(g, fam, p, 5, dt, n + 1, n, u, boundary_rule=False)
    want = np.array(u, copy=True)
    reach = np.zeros(g.shape, dtype=bool)
    flat = [cc.reshape(-1) for cc in coords]
    want = want.reshape(-1)
    a, _ = oracle.gauss_hermite(5)
    for j in range(g.size):
        x = np.array([flat[m][j] for m in range(g.dim)])
        b, s = oracle.coefficients(fam, p, g.dim, n * dt, x)
        want[j] = 0.25 + c @ (x + b * dt)
        ext = abs(s[0, 0]) * math.sqrt(2 * dt) * a.max() + np.abs(b) * dt
        ok = np.all(x - ext > np.array(g.lo)) and np.all(x + ext < np.array(g.hi))
        reach.reshape(-1)[j] = ok
    assert reach.sum() > g.size // 2
    np.testing.assert_allclose(un.reshape(-1)[reach.reshape(-1)], want[reach.reshape(-1)], atol=1e-13)


def _slopes_indep(u, h, axis):
    """Eq. (e300) with its end rule, written along one numpy axis."""
    u = np.moveaxis(u, axis, -1)
    dlt = np.diff(u, axis=-1) / h
    # node 0: (delta_0, delta_1); node i: (delta_{i-1}, delta_i);
    # node n-1: (delta_{n-2}, delta_{n-3})
    left = np.concatenate([dlt[..., :1], dlt[..., :-1], dlt[..., -1:]], axis=-1)
    right = np.concatenate([dlt[..., 1:2], dlt[..., 1:], dlt[..., -2:-1]], axis=-1)
    same = left * right > 0
    safe_l = np.where(same, left, 1.0)
    safe_r = np.where(same, right, 1.0)
    d = np.where(same, 2.0 / (1.0 / safe_l + 1.0 / safe_r), 0.0)
    return np.moveaxis(d, -1, axis)


def _cardinal(xn, h, x):
    r = abs(x - xn) / h
    if r >= 1.0:
        return 0.0, 0.0
    return 1 - 3 * r * r + 2 * r ** 3, (x - xn) * (1 - r) ** 2


def test_dense_matrix_form_2d(oracle):
    """u^n = Q Psi F u^{n+1} + (exit weights), then boundary nodes <- 1."""
    rng = np.random.default_rng(2)
    g = oracle.Grid((5, 5), (0.0, 0.0), (2.0, 1.0))
    p = [1.0, 0.2, 2 * math.pi, 0.05]
    dt, q, n = 0.01, 3, 3
    u = rng.uniform(0, 1, g.shape)
    hx, hy = g.h(0), g.h(1)
    ux = _slopes_indep(u, hx, axis=1)
    uy = _slopes_indep(u, hy, axis=0)
    J = g.size
    vec = np.concatenate([u.reshape(-1), ux.reshape(-1), uy.reshape(-1)])
    a, w = oracle.gauss_hermite(q)
    xs, ys = g.axis(0), g.axis(1)
    Psi = np.zeros((J * q * q, 3 * J))
    exit_row = np.zeros(J * q * q)
    Qm = np.zeros((J, J * q * q))
    for j in range(J):
        i, k = j % 5, j // 5
        b, s = oracle.coefficients(oracle.CELLULAR_FLOW, p, 2, n * dt, [xs[i], ys[k]])
        for qy in range(q):
            for qx in range(q):
                r = j * q * q + qy * q + qx
                Qm[j, r] = w[qx] * w[qy]
                zx = xs[i] + b[0] * dt + s[0, 0] * math.sqrt(2 * dt) * a[qx]
                zy = ys[k] + b[1] * dt + s[1, 1] * math.sqrt(2 * dt) * a[qy]
                if not (0.0 <= zx <= 2.0 and 0.0 <= zy <= 1.0):
                    exit_row[r] = 1.0
                    continue
                for kk in range(5):
                    vy, dy = _cardinal(ys[kk], hy, zy)
                    for ii in range(5):
                        vx, dx = _cardinal(xs[ii], hx, zx)
                        c = kk * 5 + ii
                        Psi[r, c] = vx * vy
                        Psi[r, J + c] = dx * vy
                        Psi[r, 2 * J + c] = vx * dy
    want = Qm @ (Psi @ vec + exit_row)
    want = want.reshape(g.shape)
    want[0, :] = want[-1, :] = 1.0
    want[:, 0] = want[:, -1] = 1.0
    got = oracle.march(g, oracle.CELLULAR_FLOW, p, q, dt, n + 1, n, u)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_dense_matrix_form_3d(oracle):
    """The same matrix form in 3D: every column of Psi is a product of three
    1D cardinal functions, with a node's value or one of its three first
    partials (Eq. (Lag11) carries no mixed partials)."""
    rng = np.random.default_rng(4)
    n = (5, 4, 4)
    g = oracle.Grid(n, (0.0, -1.0, 0.0), (2.0, 1.0, 1.5))
    p = [0.4, -0.3, 0.2, 0.6]
    dt, q = 0.01, 3
    u = rng.uniform(0, 1, g.shape)  # (nz, ny, nx)
    h = [g.h(m) for m in range(3)]
    du = [_slopes_indep(u, h[0], axis=2), _slopes_indep(u, h[1], axis=1),
          _slopes_indep(u, h[2], axis=0)]
    a, w = oracle.gauss_hermite(q)
    ax = [g.axis(m) for m in range(3)]
    want = np.zeros(g.shape)
    for l in range(n[2]):
        for k in range(n[1]):
            for i in range(n[0]):
                x = (ax[0][i], ax[1][k], ax[2][l])
                acc = 0.0
                for r in range(q):
                    for qq in range(q):
                        for pp in range(q):
                            z = [x[m] + p[m] * dt + p[3] * math.sqrt(2 * dt) * a[(pp, qq, r)[m]]
                                 for m in range(3)]
                            wt = w[pp] * w[qq] * w[r]
                            if not all(g.lo[m] <= z[m] <= g.hi[m] for m in range(3)):
                                acc += wt
                                continue
                            val = 0.0
                            for ll in range(n[2]):
                                vz, dz = _cardinal(ax[2][ll], h[2], z[2])
                                if vz == 0.0 and dz == 0.0:
                                    continue
                                for kk in range(n[1]):
                                    vy, dy = _cardinal(ax[1][kk], h[1], z[1])
                                    for ii in range(n[0]):
                                        vx, dx = _cardinal(ax[0][ii], h[0], z[0])
                                        c = (ll, kk, ii)
                                        val += (vx * vy * vz * u[c] + dx * vy * vz * du[0][c]
                                                + vx * dy * vz * du[1][c]
                                                + vx * vy * dz * du[2][c])
                            acc += wt * val
                want[l, k, i] = acc
    want[0], want[-1] = 1.0, 1.0
    want[:, 0], want[:, -1] = 1.0, 1.0
    want[:, :, 0], want[:, :, -1] = 1.0, 1.0
    got = oracle.march(g, oracle.CONST_DRIFT, p, q, dt, 1, 0, u)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_dense_matrix_form_1d(oracle):
    rng = np.random.default_rng(3)
    g = oracle.Grid((9,), (-1.0,), (1.0,))
    dt, q = 0.004, 4
    p = [0.5, 0, 0, 1.0]
    u = rng.uniform(0, 1, 9)
    h = g.h(0)
    du = _slopes_indep(u, h, axis=0)
    a, w = oracle.gauss_hermite(q)
    xs = g.axis(0)
    want = np.zeros(9)
    for j in range(9):
        acc = 0.0
        for qq in range(q):
            z = xs[j] + 0.5 * dt + math.sqrt(2 * dt) * a[qq]
            if not (-1.0 <= z <= 1.0):
                acc += w[qq]
                continue
            val = 0.0
            for i in range(9):
                v, d = _cardinal(xs[i], h, z)
                val += v * u[i] + d * du[i]
            acc += w[qq] * val
        want[j] = acc
    want[0] = want[-1] = 1.0
    got = oracle.march(g, oracle.CONST_DRIFT, p, q, dt, 1, 0, u)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_boundary_nodes_held_at_one(oracle):
    g = oracle.Grid((11, 9), (0.0, 0.0), (2.0, 1.0))
    u = oracle.march(g, oracle.CELLULAR_FLOW, [1.0, 0.2, 2 * math.pi, 1e-3], 4, 1e-3, 5, 0)
    assert np.all(u[0, :] == 1.0) and np.all(u[-1, :] == 1.0)
    assert np.all(u[:, 0] == 1.0) and np.all(u[:, -1] == 1.0)
