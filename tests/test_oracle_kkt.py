"""Pins of the oracle's KKT system and cached inverse (Eq. kkt_step_x, Remarks 1-2).

* K K^-1 = I and both are symmetric.
* A_fc^T A_fc has the closed form (n I - 1 1^T) kron P^T P, which follows
  from every agent appearing in n-1 pairs with opposite signs (Eq. A_f).
* K^-1 has a closed form built from two agent-level 17x17 inverses
  (eigen-decomposition of n I - 1 1^T); it is compared with the dense
  inverse in the agent-interleaved ordering.
"""
import numpy as np
import pytest

import oracle as O


def _mat(n, m=50, T=5.0, rho=1.0, mask=O.BC_ALL, degree=10):
    return O.build_matrices(n, m, degree, T, 0.6, 1.2, rho, mask)


@pytest.mark.parametrize("n", [2, 3, 4, 7, 16])
def test_inverse_identity_and_symmetry(n):
    M = _mat(n, m=100 if n == 16 else 50, T=8.0 if n == 16 else 5.0)
    N = M.K.shape[0]
    assert N == n * (M.nv + M.nb)
    assert np.array_equal(M.K, M.K.T)
    err = np.abs(M.K @ M.Kinv - np.eye(N)).max()
    assert err < 1e-10, err
    assert np.abs(M.Kinv - M.Kinv.T).max() < 1e-9 * np.abs(M.Kinv).max()


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_pair_gram_closed_form(n):
    M = _mat(n)
    G = (M.A_fc.T @ M.A_fc).toarray()
    PtP = M.P.T @ M.P
    ref = np.kron(n * np.eye(n) - np.ones((n, n)), PtP)
    np.testing.assert_allclose(G, ref, atol=1e-12 * np.abs(ref).max())
    # row count: m * C(n, 2) (Sec. III-B, per-iteration complexity)
    assert M.A_fc.shape == (M.m * n * (n - 1) // 2, n * M.nv)


def _interleave_perm(n, nv, nb):
    """Index map from agent-interleaved order [c_i, nu_i]_i to [c ; nu]."""
    perm = []
    for i in range(n):
        perm += list(range(i * nv, (i + 1) * nv))
        perm += list(range(n * nv + i * nb, n * nv + (i + 1) * nb))
    return np.array(perm)


@pytest.mark.parametrize("n,rho,mask", [(4, 1.0, O.BC_ALL), (7, 1.0, O.BC_ALL),
                                        (5, 3.0, O.BC_ALL), (6, 1.0, 0b011011)])
def test_kronecker_closed_form_of_inverse(n, rho, mask):
    M = _mat(n, rho=rho, mask=mask)
    nv, nb = M.nv, M.nb
    Q1 = M.ddP.T @ M.ddP
    PtP = M.P.T @ M.P
    Z = np.zeros((nb, nb))
    K0 = np.block([[Q1, M.A.T], [M.A, Z]])
    Kn = np.block([[Q1 + rho * n * PtP, M.A.T], [M.A, Z]])
    K0i, Kni = np.linalg.inv(K0), np.linalg.inv(Kn)
    closed = np.kron(np.eye(n), Kni) + np.kron(np.ones((n, n)) / n, K0i - Kni)
    perm = _interleave_perm(n, nv, nb)
    dense = M.Kinv[np.ix_(perm, perm)]
    scale = np.abs(dense).max()
    assert np.abs(closed - dense).max() < 1e-10 * scale


def test_inverse_independent_of_boundary_values():
    """Remark 2: the KKT matrix depends on n, rho and P only, not on start/goal."""
    M1 = _mat(3)
    M2 = _mat(3)
    assert np.array_equal(M1.K, M2.K)
