"""Pins for the oracle's runaway-electron model (Sec. 4.3, Eq. (ex32d)).

Coefficients, each against a fact the physics or the mathematics fixes:
* the Chandrasekhar function: C_A -> 2 nu v_T^2 / (3 sqrt(pi)) as p -> 0 and
  C_A -> nu v_T^2 / (2 p^3) for large p (delta = 0);
* the chain rule inside the p drift: b_p + C_F at xi = 1 (E = 0) equals a
  central difference of p^2 C_A, divided by p^2;
* pitch-angle scattering is a divergence-form operator: with E = 0 and no
  radiation, b_xi = (1/2) d(sigma_xi^2)/d xi; the r drift beyond V(r) is
  (1/2) d(sigma_r^2)/dr;
* without collisions and radiation the guiding-centre motion conserves the
  perpendicular momentum p sqrt(1 - xi^2) and accelerates the parallel one,
  p xi, at the rate E.

The march:
* with E = 0 the problem is even in xi, and so is the march (to rounding);
* against Monte Carlo of the SDE (Euler-Maruyama, the same face rules:
  exit value 1 at p_max, 0 at p_min and r = 1, mirror at xi = +-1 and
  r = 0): the gap shrinks under refinement at every starting point, and
  the runaway probability is near 1 where the electron is carried over
  p_max and near 0 where it is carried away from it.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

P = (3.0, 50.0, 1.0, 0.042, 1.0, 1.0, 0.5, 0.05, 20.0, 0.05, 0.02)
LO, HI = (2.0, -1.0, 0.0), (12.0, 1.0, 1.0)


def _coef(oracle, params, x):
    b, s = oracle.coefficients(oracle.RUNAWAY, params, 3, 0.0, x)
    return b, np.diag(s)


def _with(**kw):
    names = ("E", "tau", "Z", "delta", "nu", "vT", "rD", "W", "Dp", "V0", "D0")
    p = dict(zip(names, P))
    p.update(kw)
    return [p[k] for k in names]


def test_paper_parameters_and_diagonal_sigma(oracle):
    assert oracle.RUNAWAY_PARAMS == (0.3, 1e5, 1.0, 0.042, 1.0, 1.0, 0.7, 1e-2, 20.0, 0.003, 1e-4)
    _, s = oracle.coefficients(oracle.RUNAWAY, oracle.RUNAWAY_PARAMS, 3, 0.0, [10.0, 0.3, 0.5])
    assert np.count_nonzero(s - np.diag(np.diag(s))) == 0


def test_chandrasekhar_limits(oracle):
    p = _with(delta=0.0)
    _, s = _coef(oracle, p, [1e-4, 0.0, 0.5])
    assert s[0] ** 2 / 2 == pytest.approx(2.0 / (3.0 * math.sqrt(math.pi)), rel=1e-6)
    for mom in (30.0, 60.0):
        _, s = _coef(oracle, p, [mom, 0.0, 0.5])
        assert s[0] ** 2 / 2 == pytest.approx(1.0 / (2.0 * mom ** 3), rel=1e-9)


def test_p_drift_chain_rule(oracle):
    p = _with(E=0.0)
    for mom in (2.0, 3.7, 11.0, 24.0, 47.0):
        b, s = _coef(oracle, p, [mom, 1.0, 0.5])
        gam = math.sqrt(1 + (0.042 * mom) ** 2)
        ca = s[0] ** 2 / 2
        cf = 2.0 * (ca * (mom / gam))  # C_F = 2 nu v_T psi, psi = C_A y / (nu v_T^2)

        def p2ca(q):
            return q * q * _coef(oracle, p, [q, 1.0, 0.5])[1][0] ** 2 / 2

        h = 1e-4 * mom
        fd = (p2ca(mom + h) - p2ca(mom - h)) / (2 * h)
        assert b[0] + cf == pytest.approx(fd / mom ** 2, rel=1e-6, abs=1e-12)


def test_divergence_form_drifts(oracle):
    p = _with(E=0.0, tau=1e300)
    for mom, xi, r in ((2.5, 0.3, 0.2), (7.0, -0.8, 0.52), (11.0, 0.95, 0.47)):
        b, _ = _coef(oracle, p, [mom, xi, r])
        h = 1e-6

        def s2(k, x):
            return _coef(oracle, p, x)[1][k] ** 2

        dxi = (s2(1, [mom, xi + h, r]) - s2(1, [mom, xi - h, r])) / (2 * h)
        assert b[1] == pytest.approx(0.5 * dxi, rel=1e-6, abs=1e-12)
        dr = (s2(2, [mom, xi, r + h]) - s2(2, [mom, xi, r - h])) / (2 * h)
        v = 0.05 if r > 0.5 else 0.0
        assert b[2] - v == pytest.approx(0.5 * dr, rel=1e-5, abs=1e-12)


def test_collisionless_invariants(oracle):
    p = _with(nu=0.0, tau=1e300, E=0.7)
    for mom, xi in ((3.0, 0.2), (9.0, -0.6), (20.0, 0.9)):
        b, s = _coef(oracle, p, [mom, xi, 0.3])
        assert np.allclose(s[:2], 0.0)
        # d/dt (p xi) = E,  d/dt (p^2 (1 - xi^2)) = 0
        assert b[0] * xi + mom * b[1] == pytest.approx(0.7, rel=1e-12)
        assert 2 * mom * (1 - xi * xi) * b[0] - 2 * mom * mom * xi * b[1] == pytest.approx(
            0.0, abs=1e-12)


def test_even_in_xi_without_field(oracle):
    g = oracle.Grid((17, 21, 9), LO, HI)
    u = oracle.march(g, oracle.RUNAWAY, _with(E=0.0), 3, 0.05, 10, 0, nthreads=4)
    assert np.abs(u - u[:, ::-1, :]).max() <= 1e-13
    assert u[..., -1].min() == 1.0 and u[..., 0].max() == 0.0  # p_max holds 1, p_min 0
    assert u[-1, :, :-1].max() == 0.0  # the wall r = 1 holds 0 (p_max nodes excepted)


def _mc(x0, T, dt, npaths, seed):
    """Euler-Maruyama of Eq. (ex32d) with the exit checked at the t_n; the
    coefficients are written here independently (the derivative of p^2 C_A
    by a central difference)."""
    E, tau, Z, delta, nu, vT, rD, Wr, Dp, V0, D0 = P
    rng = np.random.default_rng(seed)

    def ca_of(q):
        g = np.sqrt(1 + (delta * q) ** 2)
        y = q / g
        psi = (erf(y) - y * 2 / math.sqrt(math.pi) * np.exp(-y * y)) / (2 * y * y)
        return psi, y, g

    x = np.tile(np.asarray(x0, dtype=float), (npaths, 1))
    alive = np.ones(npaths, dtype=bool)
    val = np.zeros(npaths)
    for _ in range(int(round(T / dt))):
        idx = np.nonzero(alive)[0]
        if idx.size == 0:
            break
        mom, xi, r = x[idx, 0], x[idx, 1], x[idx, 2]
        psi, y, gam = ca_of(mom)
        CA = nu * vT ** 2 * psi / y
        CB = 0.5 * nu * vT ** 2 / y * (Z + erf(y) - psi + 0.5 * y * y * delta ** 4)
        CF = 2 * nu * vT * psi
        hh = 1e-5 * mom
        f = [(mom + s * hh) ** 2 * nu * vT ** 2 * ca_of(mom + s * hh)[0] / ca_of(mom + s * hh)[1]
             for s in (1, -1)]
        dp2 = (f[0] - f[1]) / (2 * hh)
        om = 1 - xi * xi
        th = np.tanh((r - rD) / Wr)
        ep = np.exp(-(mom / Dp) ** 2)
        D = 0.5 * D0 * (1 + th) * ep
        drift = (E * xi - gam * mom / tau * om - CF + dp2 / mom ** 2,
                 E * om / mom - xi * om / (tau * gam) - 2 * xi * CB / mom ** 2,
                 np.where(r > rD, V0, 0.0) + 0.5 * D0 * (1 - th * th) / Wr * ep)
        sig = (np.sqrt(2 * CA), np.sqrt(2 * CB * np.maximum(om, 0.0)) / mom, np.sqrt(2 * D))
        z = rng.standard_normal((idx.size, 3))
        for m in range(3):
            x[idx, m] += drift[m] * dt + sig[m] * math.sqrt(dt) * z[:, m]
        x[idx, 1] = np.where(x[idx, 1] > 1, 2 - x[idx, 1], x[idx, 1])
        x[idx, 1] = np.where(x[idx, 1] < -1, -2 - x[idx, 1], x[idx, 1])
        x[idx, 2] = np.abs(x[idx, 2])
        up = x[idx, 0] > HI[0]
        gone = up | (x[idx, 0] < LO[0]) | (x[idx, 2] > HI[2])
        val[idx[up]] = 1.0
        alive[idx[gone]] = False
    return val.mean(), val.std() / math.sqrt(npaths)


def test_march_against_monte_carlo(oracle):
    """E = 3, radiation time 50, p in (2, 12), T = 3 (150 steps of 0.02),
    3 points per axis.  Starting nodes on both meshes: a likely runaway, a
    sure non-runaway, a partial one, and one on the reflecting face r = 0.
    Gaps measured: 0.043, 9e-6, 0.50, 0.012 on 21x17x11 and 0.012, 5e-5,
    0.094, 0.0026 on 41x33x21."""
    T, dt = 3.0, 0.02
    starts = [(8.0, 0.5, 0.5), (6.0, 0.0, 0.7), (5.0, 0.75, 0.5), (4.0, 0.5, 0.0)]
    mc = [_mc(x0, T, dt, 20000, 11 + k) for k, x0 in enumerate(starts)]
    gaps = []
    for n in ((21, 17, 11), (41, 33, 21)):
        g = oracle.Grid(n, LO, HI)
        u = oracle.march(g, oracle.RUNAWAY, list(P), 3, dt, int(round(T / dt)), 0, nthreads=8)
        row = []
        for x0, (m, _) in zip(starts, mc):
            ii = [int(round((x0[k] - LO[k]) / ((HI[k] - LO[k]) / (n[k] - 1)))) for k in range(3)]
            assert all(abs(g.axis(k)[ii[k]] - x0[k]) < 1e-12 for k in range(3))
            row.append(abs(u[ii[2], ii[1], ii[0]] - m))
        gaps.append(row)
    print("runaway oracle vs MC gaps (coarse, fine):", gaps)
    # from (8, 0.5, 0.5) the electron runs away unless the radial transport
    # (steepest at r_D = 0.5) carries it to the wall first: MC 0.90
    assert mc[0][0] > 0.85 and mc[1][0] < 0.01 and 0.5 < mc[2][0] < 0.95
    for k in range(len(starts)):
        assert gaps[1][k] <= 0.5 * gaps[0][k] + 4 * mc[k][1] + 1e-3, (k, gaps)
    assert max(gaps[1]) < 0.12, gaps


def test_step_face_rules_directly(oracle):
    """One step at nodes next to every face, written out point by point from
    the oracle's interpolant (pinned on its own): a point beyond xi = +-1 or
    r = 0 is mirrored into the box, one beyond p_max takes 1, one beyond
    p_min or r = 1 takes 0 (1 when it is also beyond p_max)."""
    rng = np.random.default_rng(7)
    n = (21, 17, 7)
    g = oracle.Grid(n, LO, HI)
    u = rng.uniform(0.0, 1.0, g.shape)
    dt, q = 0.3, 4
    crossed = {"xi+": 0, "xi-": 0, "r0": 0, "pmax": 0, "pmin": 0, "r1": 0}
    a, w = oracle.gauss_hermite(q)
    for E in (3.0, -3.0):  # the field drives the points over both xi faces and both p faces
        # a wide radial spread, so that r = 0 and r = 1 are crossed
        _face_rule_nodes(oracle, g, n, u, _with(E=E, D0=0.3, W=0.3), dt, q, a, w, crossed)
    assert min(crossed.values()) > 0, crossed


def _face_rule_nodes(oracle, g, n, u, params, dt, q, a, w, crossed):
    nodes, want = [], []
    for k in (0, 1, n[2] - 2):
        for j in (0, 1, n[1] // 2, n[1] - 2, n[1] - 1):
            for i in (1, 2, n[0] - 2):
                x = [g.axis(0)[i], g.axis(1)[j], g.axis(2)[k]]
                b, s = oracle.coefficients(oracle.RUNAWAY, params, 3, 0.0, x)
                acc = 0.0
                for r3 in range(q):
                    for r2 in range(q):
                        for r1 in range(q):
                            z = [x[m] + b[m] * dt + s[m, m] * math.sqrt(2 * dt) * a[(r1, r2, r3)[m]]
                                 for m in range(3)]
                            wt = w[r1] * w[r2] * w[r3]
                            for key, hit in (("xi+", z[1] > 1.0), ("xi-", z[1] < -1.0),
                                             ("r0", z[2] < 0.0), ("pmax", z[0] > HI[0]),
                                             ("pmin", z[0] < LO[0]), ("r1", z[2] > HI[2])):
                                crossed[key] += hit
                            if z[1] > 1.0:
                                z[1] = 2.0 - z[1]
                            if z[1] < -1.0:
                                z[1] = -2.0 - z[1]
                            if z[2] < 0.0:
                                z[2] = -z[2]
                            if z[0] > HI[0]:
                                acc += wt
                            elif z[0] < LO[0] or z[2] > HI[2]:
                                pass
                            else:
                                acc += wt * oracle.interp(g, u, np.array([z]))[0]
                nodes.append((k * n[1] + j) * n[0] + i)
                want.append(acc)
    got = oracle.step_nodes(g, oracle.RUNAWAY, params, q, dt, 0, u, np.array(nodes))
    np.testing.assert_allclose(got, want, atol=1e-14)


# ------------------------------------------------ the thermal-quench variant

QUENCH = (0.1, 6000.0, 1.0, 3.0, 0.005, 3.0, 0.5, 0.0, 1e-4, 2.0, 0.0, 0.01, 511.0)


def test_quench_schedule_limits(oracle):
    """At t = 0 with T0 = Ttilde the model is in its normalised units
    (v_T = nu_ee = 1, E = E_0, delta = sqrt(2 T0 / mc2)); long after the
    quench T = Tf; the temperature falls monotonically in between."""
    p0 = oracle.quench_params(QUENCH, 0.0)
    assert p0[0] == pytest.approx(0.1, rel=1e-15) and p0[5] == pytest.approx(1.0, rel=1e-15)
    assert p0[4] == pytest.approx(1.0, rel=1e-15)
    assert p0[3] == pytest.approx(math.sqrt(6.0 / 511.0), rel=1e-15)
    assert list(p0[[1, 2, 6, 7, 8, 9, 10]]) == [6000.0, 1.0, 0.0, 1e-4, 2.0, 0.0, 0.01]
    late = oracle.quench_params(QUENCH, 60.0)  # 120 cooling times
    Tf = 0.005
    assert late[5] == pytest.approx(math.sqrt(Tf / 3.0), rel=1e-12)
    assert late[0] == pytest.approx(0.1 * (3.0 / Tf) ** 1.5, rel=1e-12)
    assert late[3] == pytest.approx(math.sqrt(2 * Tf / 511.0), rel=1e-12)
    vt = [oracle.quench_params(QUENCH, t)[5] for t in np.linspace(0, 5, 41)]
    assert all(a > b for a, b in zip(vt, vt[1:]))


def test_quench_step_uses_t_n(oracle):
    """Step n of the quench variant is the static model's step with the
    constants of t_n = n dt: the same numbers, node by node."""
    g = oracle.Grid((13, 9, 7), (2.0, -1.0, 0.0), (8.0, 1.0, 1.0))
    u = np.random.default_rng(3).uniform(0, 1, g.shape)
    dt = 0.02
    for n in (0, 7, 30):
        got = oracle.march(g, oracle.RUNAWAY_QUENCH, list(QUENCH), 3, dt, n + 1, n, u)
        want = oracle.march(g, oracle.RUNAWAY, list(oracle.quench_params(QUENCH, n * dt)), 3, dt,
                            n + 1, n, u)
        assert np.array_equal(got, want), n


def test_quench_without_cooling_is_static(oracle):
    """With t_star -> infinity the temperature stays at T0 and the quench
    march is the static march with the t = 0 constants."""
    q = list(QUENCH)
    q[6] = 1e300
    g = oracle.Grid((13, 9, 7), (2.0, -1.0, 0.0), (8.0, 1.0, 1.0))
    a = oracle.march(g, oracle.RUNAWAY_QUENCH, q, 3, 0.02, 15, 0, nthreads=4)
    b = oracle.march(g, oracle.RUNAWAY, list(oracle.quench_params(q, 0.0)), 3, 0.02, 15, 0,
                     nthreads=4)
    assert np.abs(a - b).max() <= 1e-14
    # with cooling the answer moves away from the frozen one
    c = oracle.march(g, oracle.RUNAWAY_QUENCH, list(QUENCH), 3, 0.02, 15, 0, nthreads=4)
    assert np.abs(c - b).max() > 1e-3
