"""Pins of the oracle's trajectory basis (Eq. param, Sec. III-B).

The Bernstein basis is checked against facts that do not depend on the
oracle's own formulas: partition of unity, linear precision, endpoint
interpolation, closed-form values at tau = 1/2 and at the endpoints, and
derivatives taken symbolically with numpy.polynomial.
"""
import json
import os
from math import comb

import numpy as np
import pytest
from numpy.polynomial import Polynomial

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N,m,T", [(10, 50, 5.0), (10, 100, 8.0), (7, 13, 2.5), (5, 6, 1.0)])
def test_partition_of_unity_and_derivative_sums(N, m, T):
    P, dP, ddP = O.bernstein_basis(N, m, T)
    assert P.shape == (m, N + 1)
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dP.sum(1), 0.0, atol=1e-11)
    np.testing.assert_allclose(ddP.sum(1), 0.0, atol=1e-9)
    assert np.all(P >= 0)


@pytest.mark.parametrize("N,m,T", [(10, 50, 5.0), (10, 100, 8.0)])
def test_endpoint_interpolation_and_linear_precision(N, m, T):
    P, _, _ = O.bernstein_basis(N, m, T)
    e0 = np.zeros(N + 1); e0[0] = 1
    eN = np.zeros(N + 1); eN[-1] = 1
    assert np.array_equal(P[0], e0)
    assert np.array_equal(P[-1], eN)
    # sum_k (k/N) B_k(tau) = tau (linear precision of the Bernstein basis)
    tau = np.arange(m) / (m - 1)
    np.testing.assert_allclose(P @ (np.arange(N + 1) / N), tau, atol=1e-13)


def _symbolic_basis(N, k):
    t = Polynomial([0.0, 1.0])
    return comb(N, k) * t ** k * (1 - t) ** (N - k)


@pytest.mark.parametrize("N,m,T", [(10, 50, 5.0), (10, 100, 8.0), (6, 9, 3.0)])
def test_derivatives_match_symbolic_differentiation(N, m, T):
    P, dP, ddP = O.bernstein_basis(N, m, T)
    tau = np.arange(m) / (m - 1)
    for k in range(N + 1):
        b = _symbolic_basis(N, k)
        # power-form evaluation of a Bernstein polynomial loses a few digits
        np.testing.assert_allclose(P[:, k], b(tau), atol=1e-11)
        np.testing.assert_allclose(dP[:, k], b.deriv(1)(tau) / T, atol=1e-9)
        np.testing.assert_allclose(ddP[:, k], b.deriv(2)(tau) / T ** 2, atol=1e-7)


def test_golden_closed_forms():
    """Textbook closed forms stored in tests/golden/bernstein_closed_forms.json."""
    with open(os.path.join(GOLDEN, "bernstein_closed_forms.json")) as f:
        g = json.load(f)
    N = g["degree"]
    m = 3  # samples tau = 0, 1/2, 1
    P, dP, ddP = O.bernstein_basis(N, m, 1.0)
    np.testing.assert_allclose(P[1], np.array(g["B_at_half"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(dP[0], np.array(g["dB_at_0"]), atol=1e-12)
    np.testing.assert_allclose(dP[-1], np.array(g["dB_at_1"]), atol=1e-12)
    np.testing.assert_allclose(ddP[0], np.array(g["d2B_at_0"]), atol=1e-10)
    np.testing.assert_allclose(ddP[-1], np.array(g["d2B_at_1"]), atol=1e-10)


def test_boundary_rows_select_by_mask():
    P, dP, ddP = O.bernstein_basis(10, 50, 5.0)
    A = O.boundary_rows(P, dP, ddP)
    np.testing.assert_array_equal(A, np.stack([P[0], dP[0], ddP[0], P[-1], dP[-1], ddP[-1]]))
    A2 = O.boundary_rows(P, dP, ddP, 0b001001)
    np.testing.assert_array_equal(A2, np.stack([P[0], P[-1]]))
