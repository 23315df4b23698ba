"""Pins of the oracle's x/y/z QP steps (Eqs. step_x_3d-step_z_3d, cost_step_x,
eq_step_x, kkt_step_x).

The oracle solves each QP through its cached KKT inverse.  Here the same
QP is solved independently: the objective is written as a stacked least-
squares problem directly from the sums of Algorithm 1 (one row per agent
sample for the smoothness term, one row per pair and sample for the
penalty term), the equality constraints are eliminated with a null-space
basis, and the reduced problem goes to a least-squares solver.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import workloads as W


def _independent_qp(P, ddP, A, n, rho, target, beq_axis):
    """argmin 1/2 sum_i,t xdd_i(t)^2 + rho/2 sum_{i<j,t} (x_i(t)-x_j(t)-target_ij(t))^2
    subject to A c_i = b_eq,i, written from the sums themselves.

    The smoothness weight 1/2 is the one of Eq. (cost_step_x) (1/2 c^T Q_x c
    with Q_x = blockdiag(Pddot^T Pddot)); Algorithm 1 prints the sum without
    the 1/2, and the matrix form is the reading taken."""
    m, nv = P.shape
    rows, rhs = [], []
    for i in range(n):                       # smoothness rows, weight 1 under the common 1/2
        for t in range(m):
            r = np.zeros(n * nv)
            r[i * nv:(i + 1) * nv] = ddP[t]
            rows.append(r)
            rhs.append(0.0)
    q = 0
    for i in range(n):
        for j in range(i + 1, n):
            for t in range(m):
                r = np.zeros(n * nv)
                r[i * nv:(i + 1) * nv] = P[t]
                r[j * nv:(j + 1) * nv] = -P[t]
                rows.append(np.sqrt(rho) * r)
                rhs.append(np.sqrt(rho) * target[q * m + t])
            q += 1
    Ms = np.array(rows)
    rs = np.array(rhs)
    nb = A.shape[0]
    Aeq = np.zeros((n * nb, n * nv))
    for i in range(n):
        Aeq[i * nb:(i + 1) * nb, i * nv:(i + 1) * nv] = A
    c_p = np.linalg.lstsq(Aeq, beq_axis, rcond=None)[0]
    Z = sla.null_space(Aeq)
    y = np.linalg.lstsq(Ms @ Z, rs - Ms @ c_p, rcond=None)[0]
    return c_p + Z @ y


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2)])
def test_qp_step_matches_independent_least_squares(n, seed):
    rng = np.random.default_rng(seed)
    m, T = 20, 4.0
    M = O.build_matrices(n, m, 10, T, 0.6, 1.2, 1.0)
    p = n * (n - 1) // 2
    bfc = rng.standard_normal((3, p * m))
    start = rng.uniform(-2, 2, (n, 3))
    goal = rng.uniform(-2, 2, (n, 3))
    beq = O.boundary_values(start, goal)
    xi = O.qp_step(M, bfc, beq)
    for ax in range(3):
        ref = _independent_qp(M.P, M.ddP, M.A, n, M.rho, bfc[ax], beq[ax])
        np.testing.assert_allclose(xi[ax], ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_qp_step_kkt_optimality_and_boundary_exactness():
    rng = np.random.default_rng(5)
    n, m = 5, 30
    M = O.build_matrices(n, m, 10, 5.0, 0.6, 1.2, 2.0)
    bfc = rng.standard_normal((3, n * (n - 1) // 2 * m))
    beq = O.boundary_values(rng.uniform(-3, 3, (n, 3)), rng.uniform(-3, 3, (n, 3)))
    xi = O.qp_step(M, bfc, beq)
    H = M.Q + M.rho * (M.A_fc.T @ M.A_fc).toarray()
    for ax in range(3):
        c = xi[ax]
        grad = H @ c - M.rho * (M.A_fc.T @ bfc[ax])
        # stationarity: grad + A_eq^T nu = 0 for some nu
        nu = np.linalg.lstsq(M.A_eq.T, -grad, rcond=None)[0]
        assert np.abs(grad + M.A_eq.T @ nu).max() < 1e-8 * max(1.0, np.abs(grad).max())
        assert np.abs(M.A_eq @ c - beq[ax]).max() < 1e-11


def test_increment_form_equals_direct_form():
    rng = np.random.default_rng(7)
    n, m = 6, 40
    M = O.build_matrices(n, m, 10, 5.0, 0.6, 1.2, 1.0)
    bfc = rng.standard_normal((3, n * (n - 1) // 2 * m))
    beq = O.boundary_values(rng.uniform(-3, 3, (n, 3)), rng.uniform(-3, 3, (n, 3)))
    xi0 = rng.standard_normal((3, n * M.nv))
    direct = O.qp_step(M, bfc, beq)
    inc = O.qp_step_increment(M, bfc, beq, xi0)
    np.testing.assert_allclose(inc, direct, atol=1e-10 * np.abs(direct).max())


def test_initial_trajectories_are_straight_segments():
    """With zero end velocities/accelerations the smoothness-only solution is
    the same scalar profile phi(t) on every axis (the problem is linear and
    separable), so each agent moves along the straight start-goal segment."""
    p = W.box16(3)
    M = O.build_matrices(p.n, p.m, p.degree, p.T, p.a, p.b, p.rho)
    beq = O.boundary_values(p.start, p.goal)
    xi = O.initial_trajectories(M, beq)
    X = O.positions(M, xi)                           # (3, n, m)
    s = p.start.astype(np.float64).T[:, :, None]
    g = p.goal.astype(np.float64).T[:, :, None]
    dvec = g - s
    phi = np.einsum("ant,an->nt", X - s, dvec[:, :, 0]) / np.sum(dvec[:, :, 0] ** 2, 0)[:, None]
    np.testing.assert_allclose(X, s + dvec * phi[None], atol=1e-10)
    np.testing.assert_allclose(phi[:, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(phi[:, -1], 1.0, atol=1e-12)
    # all agents share one profile
    np.testing.assert_allclose(phi, np.broadcast_to(phi[0], phi.shape), atol=1e-10)
