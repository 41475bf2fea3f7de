"""Pins for the oracle's Gauss-Hermite rule (Eq. (quad), density of Eq. (expec)).

The rule is pinned to a printed textbook table, to closed forms of the
moments of the density pi^{-1/2} exp(-xi^2), to the Q = 3 closed form and to
an independent library routine.  Remark 1 (Sec. 3.1.4) uses Q* points per
dimension; the weights are normalised so that they sum to 1.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gauss_hermite_as_25_10.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, x, w = line.split()
        rows.setdefault(int(n), []).append((float(x), float(w)))
    return rows


def test_matches_printed_table(oracle):
    for n, entries in _table().items():
        a, w = oracle.gauss_hermite(n)
        for x, wt in entries:
            k = int(np.argmin(np.abs(a - x)))
            assert abs(a[k] - x) < 2e-15
            # table weights are for exp(-x^2); ours for pi^{-1/2} exp(-x^2)
            assert abs(w[k] * math.sqrt(math.pi) - wt) < 2e-15
            if x != 0.0:  # symmetric partner
                k2 = int(np.argmin(np.abs(a + x)))
                assert abs(w[k2] - w[k]) < 1e-15


def test_q3_closed_form(oracle):
    a, w = oracle.gauss_hermite(3)
    np.testing.assert_allclose(a, [-math.sqrt(1.5), 0.0, math.sqrt(1.5)], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)


@pytest.mark.parametrize("q", list(range(1, 13)))
def test_moments(q, oracle):
    """Exact for polynomials of degree <= 2q-1: E[xi^(2k)] = (2k-1)!!/2^k,
    odd moments vanish, total mass 1."""
    a, w = oracle.gauss_hermite(q)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(w > 0)
    for p in range(0, 2 * q):
        got = float(np.sum(w * a ** p))
        if p % 2:
            want = 0.0
        else:
            k = p // 2
            want = float(np.prod(np.arange(1, 2 * k, 2))) / 2 ** k if k else 1.0
        scale = float(np.sum(w * np.abs(a) ** p))
        assert abs(got - want) < 1e-13 * max(1.0, scale), (q, p, got, want)


@pytest.mark.parametrize("q", [2, 4, 6, 8, 10])
def test_against_library_routine(q, oracle):
    a, w = oracle.gauss_hermite(q)
    xa, wa = np.polynomial.hermite.hermgauss(q)
    np.testing.assert_allclose(a, xa, atol=1e-13)
    np.testing.assert_allclose(w, wa / math.sqrt(math.pi), atol=1e-14)
