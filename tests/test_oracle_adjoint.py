"""Pins for the oracle's reverse-mode derivative of the march (fko_adjoint)
against central finite differences of the oracle's own march.

L = <g, u^0> with a seeded cotangent g.  The march is differentiable away
from the kinks of the PCHIP slope rule (Eq. (e300): its branch changes where
two neighbouring differences change sign relative to each other):
* from the terminal indicator chi the parameter derivatives (A, eps, omega,
  D) match FD with h = 1e-4 (1e-4 D for D) to 1e-6 relative;
* from a random smooth terminal field (many local extrema, hence kinks
  within +-1e-4 of the base point) FD needs h = 1e-6 to stay on one branch;
  there the parameter and terminal-field derivatives match to 1e-6
  relative / 1e-8 absolute;
* the constant-drift family (b_1, b_2, s) likewise.
Interior entries of chi sit in flat data where the slope rule is
positively homogeneous but not differentiable, so FD there measures a
one-sided directional derivative; those entries are not compared.
"""
import math

import numpy as np
import pytest

import fk_inputs

G = ((41, 21), (0.0, 0.0), (2.0, 1.0))
P = [1.0, 0.3, 2 * math.pi, 0.02]
DT, N, Q = 2e-3, 15, 4


def _L(oracle, grid, fam, p, cot, u0):
    return float(np.sum(cot * oracle.march(grid, fam, p, Q, DT, N, 0, u0)))


def _fd_params(oracle, grid, fam, p, cot, u0, rel, which):
    out = {}
    for k in which:
        scale = p[3] if (fam == oracle.CELLULAR_FLOW and k == 3) else 1.0
        h = rel * scale
        pp, pm = list(p), list(p)
        pp[k] += h
        pm[k] -= h
        out[k] = (_L(oracle, grid, fam, pp, cot, u0) - _L(oracle, grid, fam, pm, cot, u0)) / (2 * h)
    return out


def test_adjoint_parameters_from_chi(oracle):
    grid = oracle.Grid(*G)
    cot = np.random.default_rng(0).standard_normal(grid.shape)
    dth, _ = oracle.adjoint(grid, oracle.CELLULAR_FLOW, P, Q, DT, N, cot)
    fd = _fd_params(oracle, grid, oracle.CELLULAR_FLOW, P, cot, None, 1e-4, range(4))
    for k in range(4):
        assert abs(dth[k] - fd[k]) <= 1e-6 * abs(fd[k]) + 1e-12, (k, dth[k], fd[k])


def test_adjoint_random_terminal_field(oracle):
    grid = oracle.Grid(*G)
    cot = np.random.default_rng(1).standard_normal(grid.shape)
    u0 = fk_inputs.random_field(grid.shape, seed=3)
    dth, dut = oracle.adjoint(grid, oracle.CELLULAR_FLOW, P, Q, DT, N, cot, u0)
    fd = _fd_params(oracle, grid, oracle.CELLULAR_FLOW, P, cot, u0, 1e-6, range(4))
    for k in range(4):
        assert abs(dth[k] - fd[k]) <= 1e-6 * abs(fd[k]) + 1e-10, (k, dth[k], fd[k])
    for idx in [(5, 7), (10, 20), (0, 3), (3, 0), (20, 40), (12, 33), (19, 1)]:
        up, um = u0.copy(), u0.copy()
        up[idx] += 1e-6
        um[idx] -= 1e-6
        fdv = (_L(oracle, grid, oracle.CELLULAR_FLOW, P, cot, up)
               - _L(oracle, grid, oracle.CELLULAR_FLOW, P, cot, um)) / 2e-6
        assert abs(dut[idx] - fdv) <= 1e-8 + 1e-6 * abs(fdv), (idx, dut[idx], fdv)


def test_adjoint_constant_drift(oracle):
    grid = oracle.Grid((31, 25), (-1.0, -1.0), (1.0, 1.0))
    p = [0.6, -0.4, 0.0, 0.35]
    cot = np.random.default_rng(2).standard_normal(grid.shape)
    u0 = fk_inputs.random_field(grid.shape, seed=9)
    dth, _ = oracle.adjoint(grid, oracle.CONST_DRIFT, p, Q, DT, N, cot, u0)
    fd = _fd_params(oracle, grid, oracle.CONST_DRIFT, p, cot, u0, 1e-6, (0, 1, 3))
    for k in (0, 1, 3):
        assert abs(dth[k] - fd[k]) <= 1e-6 * abs(fd[k]) + 1e-10, (k, dth[k], fd[k])
    assert dth[2] == 0.0  # b_3 does not exist in 2D


def test_adjoint_linear_in_cotangent(oracle):
    grid = oracle.Grid(*G)
    rng = np.random.default_rng(5)
    g1, g2 = rng.standard_normal(grid.shape), rng.standard_normal(grid.shape)
    a1, u1 = oracle.adjoint(grid, oracle.CELLULAR_FLOW, P, Q, DT, 5, g1)
    a2, u2 = oracle.adjoint(grid, oracle.CELLULAR_FLOW, P, Q, DT, 5, g2)
    a3, u3 = oracle.adjoint(grid, oracle.CELLULAR_FLOW, P, Q, DT, 5, 2 * g1 - g2)
    np.testing.assert_allclose(a3, 2 * a1 - a2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(u3, 2 * u1 - u2, rtol=1e-12, atol=1e-12)
