"""Pins of the oracle's static obstacles (Sec. IV-A; reading R-obst).

Each (agent, obstacle, sample) is one more row of A_fc with the agent's +P
and a fixed partner, the obstacle centre.  Pinned independently of the
oracle's own assembly:

* no obstacles: exactly the plain solve;
* the penalty Gram matrix is ((n + n_obs) I - 1 1^T) (x) P^T P, and the
  inverse has the two-block closed form with the agent-level matrices
  shifted by n_obs rho P^T P (eigen-decomposition of the shifted matrix);
* the QP step equals a least-squares solve written from the sums (pair
  rows and obstacle rows built by loops), equality constraints eliminated
  by a null-space basis;
* solved instances clear every obstacle (scaled distance computed here from
  the positions) and keep their boundary values, where the straight-line
  trajectories pass through the obstacle;
* mirroring the scene mirrors the solution.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import workloads as W


def _mats(prob, n_obs, rho=1.0, m=None):
    return O.build_matrices(prob.n, m or prob.m, prob.degree, prob.T, prob.a, prob.b, rho,
                            n_obs=n_obs)


def test_zero_obstacles_is_the_plain_solve():
    prob = W.random_box(5, 2, box=(5.0, 5.0, 2.5), m=30, T=4.0)
    M = _mats(prob, 0)
    ref = O.solve(M, prob.start, prob.goal, 25, mode="R2")
    st, so = O.solve_obstacles(M, prob.start, prob.goal, np.zeros((0, 5)), 25, mode="R2")
    assert np.array_equal(st.xi, ref.xi) and np.array_equal(st.lam, ref.lam)
    assert st.r_max == ref.r_max and st.k == ref.k and so.lam.shape == (3, 0)


@pytest.mark.parametrize("n,n_obs,rho", [(3, 1, 1.0), (4, 3, 1.0), (5, 2, 2.5)])
def test_gram_and_inverse_closed_forms(n, n_obs, rho):
    prob = W.random_box(n, 1, box=(5.0, 5.0, 2.5), m=40, T=5.0)
    M = _mats(prob, n_obs, rho)
    PtP = M.P.T @ M.P
    G = (M.A_fc.T @ M.A_fc + M.A_obs.T @ M.A_obs).toarray()
    ref = np.kron((n + n_obs) * np.eye(n) - np.ones((n, n)), PtP)
    np.testing.assert_allclose(G, ref, atol=1e-12 * np.abs(ref).max())
    assert M.A_obs.shape == (n * n_obs * M.m, n * M.nv)
    nv, nb = M.nv, M.nb
    Q1 = M.ddP.T @ M.ddP
    Z = np.zeros((nb, nb))
    K0 = np.block([[Q1 + rho * n_obs * PtP, M.A.T], [M.A, Z]])
    Kn = np.block([[Q1 + rho * (n + n_obs) * PtP, M.A.T], [M.A, Z]])
    K0i, Kni = np.linalg.inv(K0), np.linalg.inv(Kn)
    closed = np.kron(np.eye(n), Kni) + np.kron(np.ones((n, n)) / n, K0i - Kni)
    perm = []
    for i in range(n):
        perm += list(range(i * nv, (i + 1) * nv))
        perm += list(range(n * nv + i * nb, n * nv + (i + 1) * nb))
    dense = M.Kinv[np.ix_(perm, perm)]
    assert np.abs(closed - dense).max() < 1e-10 * np.abs(dense).max()


def _independent_qp(P, ddP, A, n, n_obs, rho, tgt_pairs, tgt_obs, beq_axis):
    """argmin 1/2 sum xdd^2 + rho/2 sum_{i<j,t} (x_i - x_j - b_ij)^2
    + rho/2 sum_{i,o,t} (x_i - b_io)^2 s.t. A c_i = b_eq,i, from the sums."""
    m, nv = P.shape
    rows, rhs = [], []
    for i in range(n):
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
                rhs.append(np.sqrt(rho) * tgt_pairs[q * m + t])
            q += 1
    for i in range(n):
        for o in range(n_obs):
            for t in range(m):
                r = np.zeros(n * nv)
                r[i * nv:(i + 1) * nv] = P[t]
                rows.append(np.sqrt(rho) * r)
                rhs.append(np.sqrt(rho) * tgt_obs[(i * n_obs + o) * m + t])
    Ms = np.array(rows)
    rs = np.array(rhs)
    nb = A.shape[0]
    Aeq = np.zeros((n * nb, n * nv))
    for i in range(n):
        Aeq[i * nb:(i + 1) * nb, i * nv:(i + 1) * nv] = A
    c_p = np.linalg.lstsq(Aeq, beq_axis, rcond=None)[0]
    Zn = sla.null_space(Aeq)
    y = np.linalg.lstsq(Ms @ Zn, rs - Ms @ c_p, rcond=None)[0]
    return c_p + Zn @ y


@pytest.mark.parametrize("n,n_obs,seed", [(2, 1, 0), (3, 2, 1)])
def test_qp_step_matches_independent_least_squares(n, n_obs, seed):
    rng = np.random.default_rng(seed)
    m, T = 20, 4.0
    M = O.build_matrices(n, m, 10, T, 0.6, 1.2, 1.5, n_obs=n_obs)
    p = n * (n - 1) // 2
    bfc = rng.standard_normal((3, p * m))
    bobs = rng.standard_normal((3, n * n_obs * m))
    start = rng.uniform(-2, 2, (n, 3))
    goal = rng.uniform(-2, 2, (n, 3))
    beq = O.boundary_values(start, goal)
    xi = O.qp_step_obstacles(M, bfc, bobs, beq)
    for ax in range(3):
        ref = _independent_qp(M.P, M.ddP, M.A, n, n_obs, M.rho, bfc[ax], bobs[ax], beq[ax])
        np.testing.assert_allclose(xi[ax], ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def _crossing_scene():
    """Four agents crossing a 6 m square through its centre, where an
    obstacle (combined semi-axes 1.0 x 1.4 m) sits on every straight path."""
    start = np.array([[-3.0, 0.2, 1.0], [3.0, -0.2, 1.0], [0.2, -3.0, 1.0], [-0.2, 3.0, 1.0]],
                     np.float32)
    goal = np.array([[3.0, -0.2, 1.0], [-3.0, 0.2, 1.0], [-0.2, 3.0, 1.0], [0.2, -3.0, 1.0]],
                    np.float32)
    obst = np.array([[0.05, 0.1, 1.0, 1.0, 1.4]], np.float32)
    return W.Problem(n=4, m=60, T=6.0, start=start, goal=goal), obst


def _scaled_distance(pos, ob):
    """min over agents and samples of the combined-spheroid norm to obstacle ob."""
    d = pos - ob[:3, None, None]                      # (3, n, m)
    return np.sqrt((d[0] ** 2 + d[1] ** 2) / ob[3] ** 2 + d[2] ** 2 / ob[4] ** 2).min()


@pytest.mark.parametrize("mode", ["R3", "R2"])
def test_solutions_clear_the_obstacle(mode):
    prob, obst = _crossing_scene()
    M0 = _mats(prob, 0)
    free = O.solve(M0, prob.start, prob.goal, 300, 1e-3, mode=mode)
    pos_free = O.positions(M0, free.xi)
    assert _scaled_distance(pos_free, obst[0].astype(np.float64)) < 0.9  # paths cross it
    M = _mats(prob, 1)
    st, so = O.solve_obstacles(M, prob.start, prob.goal, obst, 1500, 2e-3, mode=mode)
    assert st.r_max < 2e-3, st.r_max
    pos = O.positions(M, st.xi)
    assert _scaled_distance(pos, obst[0].astype(np.float64)) > 1.0 - 5e-3
    # boundary values still hold
    np.testing.assert_allclose(pos[:, :, 0].T, prob.start, atol=1e-9)
    np.testing.assert_allclose(pos[:, :, -1].T, prob.goal, atol=1e-9)
    # pairs clear each other too
    for i in range(4):
        for j in range(i + 1, 4):
            dd = pos[:, i] - pos[:, j]
            s = np.sqrt((dd[0] ** 2 + dd[1] ** 2) / prob.a ** 2 + dd[2] ** 2 / prob.b ** 2)
            assert s.min() > 1.0 - 5e-3


@pytest.mark.parametrize("mode,upper", [("R2", 1.01), ("R3", 1.2)])
def test_single_detour_touches_the_obstacle(mode, upper):
    """One agent's straight path runs through an obstacle (combined semi-axes
    1.0 x 1.4 m), the other's far from it: the detour clears the obstacle and,
    in the literal reading, touches it (the constraint is active, so its
    extents are the ones used); the lambda-free reading stops at the first
    feasible iterate, a little outside."""
    start = np.array([[-3.0, 0.2, 1.0], [-3.0, 2.8, 1.0]], np.float32)
    goal = np.array([[3.0, 0.2, 1.0], [3.0, 2.8, 1.0]], np.float32)
    obst = np.array([[0.0, 0.0, 1.0, 1.0, 1.4]], np.float32)
    prob = W.Problem(n=2, m=60, T=6.0, start=start, goal=goal)
    M = _mats(prob, 1)
    st, so = O.solve_obstacles(M, prob.start, prob.goal, obst, 1500, 1e-4, mode=mode)
    assert st.r_max < 1e-4, st.r_max
    pos = O.positions(M, st.xi)
    dmin = _scaled_distance(pos[:, :1], obst[0].astype(np.float64))
    assert 1.0 - 2e-4 < dmin < upper, dmin


def test_mirrored_scene_gives_mirrored_solution():
    prob, obst = W.obstacle_box(5, 3, 4, box=(6.0, 6.0, 3.0), m=40, T=6.0)
    M = _mats(prob, 3)
    st, _ = O.solve_obstacles(M, prob.start, prob.goal, obst, 30, mode="R2")
    ms, mg, mo = prob.start.copy(), prob.goal.copy(), obst.copy()
    ms[:, 0] *= -1
    mg[:, 0] *= -1
    mo[:, 0] *= -1
    st2, _ = O.solve_obstacles(M, ms, mg, mo, 30, mode="R2")
    xm = st2.xi.copy()
    xm[0] *= -1
    np.testing.assert_allclose(xm, st.xi, rtol=0, atol=1e-9 * np.abs(st.xi).max())
