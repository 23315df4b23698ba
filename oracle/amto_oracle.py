"""FP64 CPU oracle of the alternating-minimisation (AM) multi-agent trajectory
optimiser (Rastgar et al., arXiv 2011.04240, Section III, Algorithm 1).

TEST INFRASTRUCTURE ONLY.  This module is imported by the test-suite, by the
package smoke check and by the benchmark's CPU-baseline leg.  The product
path (the CUDA library and its Python binding) never imports, links or calls
it, and it shares no code, tables or constants with that path.

Everything is plain numpy/scipy float64, following the paper's equations in
the paper's order and notation:

  * basis P, Pdot, Pddot ............ Eq. (param), Sec. III-B
  * Q_x = blockdiag(Pddot^T Pddot) .. Sec. III-B (smoothness Hessian)
  * A, A_eq, b_eq ................... Sec. III-B (boundary conditions)
  * A_fc ............................ Eq. (A_f), stacked pair rows
  * b_fc ............................ Eq. (b_f)
  * KKT system, cached inverse ...... Eq. (kkt_step_x), Remarks 1-2
  * alpha/beta closed form .......... Eq. (sphere_project), Sec. III-C "Step (step_alpha)"
  * d step .......................... Eq. (step_d), clipped d >= 1 (Eq. alpha_beta_constr)
  * lambda update ................... Eq. (lag_update)
  * loop and stopping rule .......... Algorithm 1

Readings of ambiguous passages (each also listed in the design notes):
  R-basis   the paper leaves P open; degree-N Bernstein on tau = t/T with
            samples t_k = k T/(m-1), k = 0..m-1 (endpoints are rows 1 and m).
  R-pairs   the pair sum runs over unordered pairs i<j, rows ordered i-major
            then time, exactly the staircase of Eq. (A_f).
  R-sq      Eq. (quad_multiagent) lacks its squares; the constraint is
            (dx^2+dy^2)/l_xy^2 + dz^2/l_z^2 >= 1.
  R-rho     the QP objective is 1/2 c^T Q c + rho/2 ||A_fc c - b||^2, so the
            KKT right-hand side is [rho A_fc^T b ; b_eq] (Eq. kkt_step_x prints
            it without rho; all workloads use rho = 1).  The smoothness weight
            is that of the matrix form, 1/2 c^T Q_x c with
            Q_x = blockdiag(Pddot^T Pddot) (Algorithm 1 prints the sum of
            squared accelerations without the 1/2).
  R-beta    Delta_x / (l_xy cos alpha) in Eq. (sphere_project) equals
            hypot(Delta_x, Delta_y)/l_xy wherever cos alpha != 0; the hypot
            form is used so that cos alpha = 0 is defined.
  R-d       the d clip "[0 1]" of Sec. III-C contradicts d >= 1 of
            Eq. (alpha_beta_constr); d = max(1, d_hat), no upper bound.
  R-lambda  (mode "R2", default) alpha, beta from Delta only (Eq. sphere_project);
            the d step keeps ^k lambda / rho (Eq. step_d).
            (mode "R3") lambda enters only b_fc and the lambda update.
            (mode "R1") textbook ADMM: lambda/rho also inside the alpha/beta
            projection (oracle only).
  R-init    Algorithm 1 leaves the k=0 values open: lambda^0 = 0, xi^0 is the
            smoothness-only solution of each agent under its boundary
            conditions, and (alpha, beta, d)^0 is the projection of Delta^0
            with lambda = 0 (no lambda update).
  R-stop    loop while k < maxiter and r_max >= tol, where r_max is the
            largest Euclidean norm of f_c over all pairs and samples; the
            iteration count is the number of QP solves.
  R-degen   Delta = 0: atan2(0,0) = 0, so alpha = beta = 0.
  R-rho-sched  Sec. IV-A uses 10 increasing rho values, the larger ones in
            the later iterations, without giving the values or the switch:
            rho_j = rho_0 g^j (j = 0..J-1) and QP solve k (k >= 1) belongs to
            stage min(J-1, (k-1) div E); iteration k runs entirely with rho_k
            (the target b of Eq. b_f, the d step and the lambda update), and
            lambda carries over unchanged across a switch.
  R-obst    Sec. IV-A (static obstacles by their circumscribing spheres; only
            the cost of A_fc^T b grows with their number, linearly): every
            (agent i, obstacle o, sample t) is one more row of A_fc with +P in
            agent i's columns and a fixed partner, the obstacle centre c_o.
            Delta = x_i(t) - c_o is projected on the combined agent-obstacle
            spheroid whose semi-axes (a_o, b_o) are given per obstacle; the
            row's target is c_o + d u - lambda/rho and its lambda is updated
            like a pair's (same reading R-lambda).  rho A_fc^T A_fc gains
            n_obs rho P^T P per agent, so the cached inverse depends on
            (n, n_obs, rho).  Obstacle rows are ordered agent-major, then
            obstacle, then time; lambda^0 = 0 on them; they count in r_max.
  R-planar  Sec. III's "disks in 2D": agents in the x-y plane are disks of
            radius l_xy; Delta = (Delta_x, Delta_y), alpha = atan2(Delta_y,
            Delta_x) (0 when Delta = 0, as R-degen), u = l_xy (cos alpha,
            sin alpha), d and lambda as in 3-D.  The z axis is dropped: z
            boundary values are taken as 0, its QP has no pair term, and the
            z coefficients stay 0.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np
import scipy.sparse as sp

# Boundary-condition rows of A, in the order of Sec. III-B:
# P_1, Pdot_1, Pddot_1, P_m, Pdot_m, Pddot_m.
BC_ALL = 0x3F


# ---------------------------------------------------------------------------
# Basis and problem matrices (Sec. III-B)
# ---------------------------------------------------------------------------

def bernstein_basis(degree: int, m: int, T: float):
    """P, Pdot, Pddot of Eq. (param): m x (degree+1) basis matrices.

    B_{k,N}(tau) = C(N,k) tau^k (1-tau)^(N-k), tau = t/T, t_k = k T/(m-1).
    dB_{k,N}/dtau = N (B_{k-1,N-1} - B_{k,N-1});
    d2B_{k,N}/dtau2 = N(N-1)(B_{k-2,N-2} - 2 B_{k-1,N-2} + B_{k,N-2});
    chain rule: d/dt = (1/T) d/dtau.
    """
    N = degree
    tau = np.arange(m, dtype=np.float64) / (m - 1)

    def B(nn, k):
        if k < 0 or k > nn or nn < 0:
            return np.zeros_like(tau)
        return comb(nn, k) * tau ** k * (1.0 - tau) ** (nn - k)

    P = np.stack([B(N, k) for k in range(N + 1)], axis=1)
    dP = np.stack([N * (B(N - 1, k - 1) - B(N - 1, k)) for k in range(N + 1)], axis=1) / T
    ddP = np.stack([N * (N - 1) * (B(N - 2, k - 2) - 2.0 * B(N - 2, k - 1) + B(N - 2, k))
                    for k in range(N + 1)], axis=1) / T ** 2
    return P, dP, ddP


def boundary_rows(P, dP, ddP, bc_mask: int = BC_ALL):
    """A of Sec. III-B: first and last rows of P, Pdot, Pddot (selected by mask)."""
    rows = [P[0], dP[0], ddP[0], P[-1], dP[-1], ddP[-1]]
    return np.stack([r for i, r in enumerate(rows) if (bc_mask >> i) & 1])


def pair_list(n: int):
    """Unordered pairs (i, j), i < j, i-major: the row blocks of Eq. (A_f)."""
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def pair_matrix(P, n: int):
    """A_fc of Eq. (A_f) as a sparse (p*m) x (n*nv) matrix.

    Pair block (i, j) occupies rows [q*m, (q+1)*m) with +P in agent i's
    columns and -P in agent j's columns, so A_fc c_x stacks x_i(t) - x_j(t).
    """
    m, nv = P.shape
    blocks = []
    for (i, j) in pair_list(n):
        row = [None] * n
        row[i] = sp.csr_matrix(P)
        row[j] = sp.csr_matrix(-P)
        for k in range(n):
            if row[k] is None:
                row[k] = sp.csr_matrix((m, nv))
        blocks.append(row)
    return sp.bmat(blocks, format="csr")


@dataclasses.dataclass
class Matrices:
    n: int
    m: int
    degree: int
    T: float
    a: float
    b: float
    rho: float
    bc_mask: int
    P: np.ndarray
    dP: np.ndarray
    ddP: np.ndarray
    A: np.ndarray          # n_b x nv
    Q: np.ndarray          # (n nv) x (n nv) = blockdiag(Pddot^T Pddot)
    A_eq: np.ndarray       # (n n_b) x (n nv) = blockdiag(A)
    A_fc: sp.csr_matrix    # (p m) x (n nv)
    K: np.ndarray          # KKT matrix of Eq. (kkt_step_x)
    Kinv: np.ndarray       # its inverse (Remark 1: computed once)
    n_obs: int = 0         # static obstacles per instance (reading R-obst)
    A_obs: sp.csr_matrix | None = None   # (n n_obs m) x (n nv) agent-obstacle rows
    planar: bool = False   # disks in the x-y plane (reading R-planar)

    @property
    def nv(self):
        return self.degree + 1

    @property
    def nb(self):
        return self.A.shape[0]


def obstacle_matrix(P, n: int, n_obs: int):
    """Agent-obstacle rows of A_fc (reading R-obst) as a sparse matrix: block
    (i, o) occupies rows [(i n_obs + o) m, (i n_obs + o + 1) m) with +P in
    agent i's columns; the partner (the obstacle centre) is fixed."""
    m, nv = P.shape
    blocks = []
    for i in range(n):
        for o in range(n_obs):
            row = [sp.csr_matrix((m, nv)) for _ in range(n)]
            row[i] = sp.csr_matrix(P)
            blocks.append(row)
    if not blocks:
        return sp.csr_matrix((0, n * nv))
    return sp.bmat(blocks, format="csr")


def build_matrices(n: int, m: int, degree: int, T: float, a: float, b: float,
                   rho: float, bc_mask: int = BC_ALL, n_obs: int = 0,
                   planar: bool = False) -> Matrices:
    """Assemble Q_x, A_eq, A_fc and the KKT matrix, and invert it (Eq. kkt_step_x).

    The inverse is a dense LAPACK LU-based inverse (partial pivoting); it is
    computed once per (n, rho, P) as Remarks 1-2 state (and per obstacle
    count, reading R-obst).
    """
    P, dP, ddP = bernstein_basis(degree, m, T)
    A = boundary_rows(P, dP, ddP, bc_mask)
    Q = np.kron(np.eye(n), ddP.T @ ddP)
    A_eq = np.kron(np.eye(n), A)
    A_fc = pair_matrix(P, n)
    A_obs = obstacle_matrix(P, n, n_obs)
    H = Q + rho * (A_fc.T @ A_fc).toarray() + rho * (A_obs.T @ A_obs).toarray()
    nz = A_eq.shape[0]
    K = np.block([[H, A_eq.T], [A_eq, np.zeros((nz, nz))]])
    Kinv = np.linalg.inv(K)
    return Matrices(n, m, degree, T, a, b, rho, bc_mask, P, dP, ddP, A, Q, A_eq,
                    A_fc, K, Kinv, n_obs, A_obs, planar)


def planar_inputs(start, goal):
    """Start and goal of a planar problem (reading R-planar): z taken as 0."""
    s = np.array(start, np.float64, copy=True)
    g = np.array(goal, np.float64, copy=True)
    s[:, 2] = 0.0
    g[:, 2] = 0.0
    return s, g


def boundary_values(start, goal, bc_mask: int = BC_ALL, bc_extra=None):
    """b_eq per axis: (3, n * n_b), agent-major, rows in the order of A.

    start, goal: (n, 3).  bc_extra (optional): (n, 2, 2, 3) holding
    [t0 / T][velocity / acceleration][axis]; zero when absent.
    """
    start = np.asarray(start, np.float64)
    goal = np.asarray(goal, np.float64)
    n = start.shape[0]
    ext = np.zeros((n, 2, 2, 3)) if bc_extra is None else np.asarray(bc_extra, np.float64)
    vals = np.stack([start, ext[:, 0, 0], ext[:, 0, 1], goal, ext[:, 1, 0], ext[:, 1, 1]],
                    axis=1)                      # (n, 6, 3)
    keep = [i for i in range(6) if (bc_mask >> i) & 1]
    vals = vals[:, keep, :]                      # (n, n_b, 3)
    return np.ascontiguousarray(vals.transpose(2, 0, 1).reshape(3, -1))


# ---------------------------------------------------------------------------
# Sub-steps of Algorithm 1
# ---------------------------------------------------------------------------

def pair_differences(M: Matrices, xi):
    """Delta = A_fc c per axis: (3, p*m), xi given as (3, n*nv).

    Formed as x_i(t) - x_j(t) from the positions (Eqs. A_f, sphere_proposed),
    so agents with identical coefficients give Delta = 0 exactly and take
    the R-degen direction (a product with A_fc's +P/-P rows leaves a
    rounding residue there instead)."""
    pos = np.einsum("tk,ank->ant", M.P, np.asarray(xi, np.float64).reshape(3, M.n, M.nv))
    pl = pair_list(M.n)
    if not pl:
        return np.zeros((3, 0))
    ii = np.array([q[0] for q in pl])
    jj = np.array([q[1] for q in pl])
    return (pos[:, ii, :] - pos[:, jj, :]).reshape(3, -1)


def alpha_beta(D, a: float, b: float):
    """Closed-form alpha, beta of Eq. (sphere_project); beta clipped to [0, pi]."""
    dx, dy, dz = D
    alpha = np.arctan2(dy, dx)
    beta = np.arctan2(np.hypot(dx, dy) / a, dz / b)
    return alpha, np.clip(beta, 0.0, np.pi)


def spheroid_direction(alpha, beta, a: float, b: float):
    """(l_xy sin b cos a, l_xy sin b sin a, l_z cos b) of Eq. (sphere_proposed)."""
    return np.stack([a * np.sin(beta) * np.cos(alpha),
                     a * np.sin(beta) * np.sin(alpha),
                     b * np.cos(beta)])


def d_step(W, U):
    """Eq. (step_d): per pair-time scalar QP min_d ||W - d U||^2, clipped d >= 1."""
    d_hat = np.sum(W * U, axis=0) / np.sum(U * U, axis=0)
    return np.maximum(1.0, d_hat)


def projection(D, lam, M: Matrices, mode: str = "R2", a=None, b=None):
    """alpha, beta, d steps for all pair-times (Eqs. sphere_project, step_d).

    `a`, `b` (scalars or one value per row) replace the agents' semi-axes,
    for the agent-obstacle rows (reading R-obst)."""
    a = M.a if a is None else a
    b = M.b if b is None else b
    if mode == "R1":
        Wab = D + lam / M.rho
    else:
        Wab = D
    if getattr(M, "planar", False):  # disks (reading R-planar): the in-plane angle only
        alpha = np.arctan2(Wab[1], Wab[0])
        beta = np.full_like(alpha, np.pi / 2)
        U = np.stack([a * np.cos(alpha), a * np.sin(alpha), np.zeros_like(alpha)])
    else:
        alpha, beta = alpha_beta(Wab, a, b)
        U = spheroid_direction(alpha, beta, a, b)
    Wd = D if mode == "R3" else D + lam / M.rho
    d = d_step(Wd, U)
    return alpha, beta, d, U


def target_vector(alpha, beta, d, lam, M: Matrices, a=None, b=None):
    """b_fc of Eq. (b_f) per axis: l d sin/cos terms minus lambda/rho."""
    a = M.a if a is None else a
    b = M.b if b is None else b
    if getattr(M, "planar", False):
        U = np.stack([a * np.cos(alpha), a * np.sin(alpha), np.zeros_like(alpha)])
        return d * U - lam / M.rho
    return d * spheroid_direction(alpha, beta, a, b) - lam / M.rho


def qp_step(M: Matrices, bfc, beq):
    """x/y/z QPs of Algorithm 1 via Eq. (kkt_step_x) and the cached inverse.

    rhs = [rho A_fc^T b_fc ; b_eq] for each axis; c = (K^-1 rhs)[:n nv].
    """
    nvn = M.n * M.nv
    rhs = np.concatenate([M.rho * np.stack([M.A_fc.T @ bfc[ax] for ax in range(3)]), beq],
                         axis=1)                 # (3, n nv + n n_b)
    sol = (M.Kinv @ rhs.T).T
    return sol[:, :nvn]


def qp_step_increment(M: Matrices, bfc, beq, xi):
    """Same QP through the increment form used on the GPU (self-check only).

    xi+ = xi + K^-1_top [rho A_fc^T (b - A_fc xi) - Q xi ; b_eq - A_eq xi];
    identical to qp_step in exact arithmetic because the top block row of
    K^-1 K is [I 0].
    """
    nvn = M.n * M.nv
    D = pair_differences(M, xi)
    g = np.stack([M.rho * (M.A_fc.T @ (bfc[ax] - D[ax])) - M.Q @ xi[ax] for ax in range(3)])
    e = beq - (M.A_eq @ xi.T).T
    rhs = np.concatenate([g, e], axis=1)
    return xi + (M.Kinv[:nvn] @ rhs.T).T


def lambda_update(lam, D, d, U, rho: float):
    """Eq. (lag_update): lambda += rho (Delta - d u); also returns f_c."""
    fc = D - d * U
    return lam + rho * fc, fc


def residual_max(fc):
    """max over pairs and samples of ||f_c||_2 (Algorithm 1 stopping norm)."""
    if fc.shape[1] == 0:
        return 0.0
    return float(np.sqrt(np.max(np.sum(fc * fc, axis=0))))


def initial_trajectories(M: Matrices, beq):
    """xi^0: per agent and axis, argmin 1/2 c^T Pddot^T Pddot c s.t. A c = b_eq.

    Solved through the agent-level KKT matrix [[Pddot^T Pddot, A^T], [A, 0]].
    """
    nv, nb = M.nv, M.nb
    K0 = np.block([[M.ddP.T @ M.ddP, M.A.T], [M.A, np.zeros((nb, nb))]])
    K0inv = np.linalg.inv(K0)
    xi = np.zeros((3, M.n * nv))
    for ax in range(3):
        for i in range(M.n):
            rhs = np.concatenate([np.zeros(nv), beq[ax, i * nb:(i + 1) * nb]])
            xi[ax, i * nv:(i + 1) * nv] = (K0inv @ rhs)[:nv]
    return xi


@dataclasses.dataclass
class State:
    xi: np.ndarray       # (3, n nv)
    lam: np.ndarray      # (3, p m), pair-major then time
    alpha: np.ndarray    # (p m,)
    beta: np.ndarray
    d: np.ndarray
    r_max: float
    k: int               # number of QP solves performed


def init_state(M: Matrices, beq, mode: str = "R2") -> State:
    """k = 0 values of Algorithm 1 (reading R-init)."""
    xi = initial_trajectories(M, beq)
    D = pair_differences(M, xi)
    lam = np.zeros_like(D)
    alpha, beta, d, U = projection(D, lam, M, mode)
    return State(xi, lam, alpha, beta, d, residual_max(D - d * U), 0)


def am_iteration(M: Matrices, st: State, beq, mode: str = "R2",
                 increment: bool = False) -> State:
    """One pass of the while-body of Algorithm 1: x/y/z QPs, alpha/beta, d, lambda."""
    bfc = target_vector(st.alpha, st.beta, st.d, st.lam, M)
    if increment:
        xi = qp_step_increment(M, bfc, beq, st.xi)
    else:
        xi = qp_step(M, bfc, beq)
    D = pair_differences(M, xi)
    alpha, beta, d, U = projection(D, st.lam, M, mode)
    lam, fc = lambda_update(st.lam, D, d, U, M.rho)
    return State(xi, lam, alpha, beta, d, residual_max(fc), st.k + 1)


def solve(M: Matrices, start, goal, max_iters: int, tol: float = 0.0,
          mode: str = "R2", bc_extra=None, increment: bool = False,
          state: State | None = None, history: list | None = None) -> State:
    """Algorithm 1: iterate while k < max_iters and r_max >= tol.

    `state` warm-starts from given (xi, lambda, alpha, beta, d); `history`
    (if a list) receives r_max after every iteration.
    """
    beq = boundary_values(start, goal, M.bc_mask, bc_extra)
    st = init_state(M, beq, mode) if state is None else state
    while st.k < max_iters:
        st = am_iteration(M, st, beq, mode, increment)
        if history is not None:
            history.append(st.r_max)
        if st.r_max < tol:
            break
    return st


def rho_stage(k: int, n_stages: int, stage_iters: int) -> int:
    """Stage of QP solve k (k >= 1) in the increasing-rho schedule (R-rho-sched)."""
    return min(n_stages - 1, (k - 1) // stage_iters)


def solve_schedule(Ms: list, stage_iters: int, start, goal, max_iters: int, tol: float = 0.0,
                   mode: str = "R2", history: list | None = None) -> State:
    """Algorithm 1 with the increasing penalty of Sec. IV-A (reading
    R-rho-sched): `Ms` holds the matrices (cached inverses) of the stages in
    increasing rho; iteration k uses Ms[rho_stage(k)].  Same loop and stopping
    rule as `solve`."""
    beq = boundary_values(start, goal, Ms[0].bc_mask)
    st = init_state(Ms[0], beq, mode)
    while st.k < max_iters:
        M = Ms[rho_stage(st.k + 1, len(Ms), stage_iters)]
        st = am_iteration(M, st, beq, mode)
        if history is not None:
            history.append(st.r_max)
        if st.r_max < tol:
            break
    return st


def warm_state(M: Matrices, xi, lam, mode: str = "R2") -> State:
    """State at a given (xi, lambda): alpha, beta, d from the projection of Delta.

    Matches a solve that resumes from trajectories `xi` and multipliers
    `lam`, with (alpha, beta, d) recomputed from Delta and lam (no lambda
    update), the same way the k = 0 values are formed.
    """
    xi = np.asarray(xi, np.float64)
    lam = np.asarray(lam, np.float64)
    D = pair_differences(M, xi)
    alpha, beta, d, U = projection(D, lam, M, mode)
    return State(xi, lam, alpha, beta, d, residual_max(D - d * U), 0)


def positions(M: Matrices, xi):
    """x_i(t_k) = P c_{x_i}: (3, n, m)."""
    return np.einsum("tk,ank->ant", M.P, xi.reshape(3, M.n, M.nv))


# ---------------------------------------------------------------------------
# Static obstacles (reading R-obst)
# ---------------------------------------------------------------------------

def obstacle_rows(M: Matrices, obstacles):
    """Per agent-obstacle row (i, o, t): the centre c_o (3, rows) and the
    semi-axes a_o, b_o (rows,).  obstacles: (n_obs, 5) = (cx, cy, cz, a_o, b_o)."""
    ob = np.asarray(obstacles, np.float64).reshape(M.n_obs, 5)
    o_of_row = np.tile(np.repeat(np.arange(M.n_obs), M.m), M.n)
    return ob[o_of_row, :3].T.copy(), ob[o_of_row, 3].copy(), ob[o_of_row, 4].copy()


def obstacle_differences(M: Matrices, xi, C):
    """Delta = x_i(t) - c_o per axis: (3, n n_obs m)."""
    return np.stack([M.A_obs @ xi[ax] for ax in range(3)]) - C


@dataclasses.dataclass
class ObstacleState:
    lam: np.ndarray      # (3, n n_obs m)
    alpha: np.ndarray
    beta: np.ndarray
    d: np.ndarray
    r_max: float


def qp_step_obstacles(M: Matrices, bfc, bobs, beq):
    """QP of Eq. (kkt_step_x) with the agent-obstacle rows stacked under the
    pair rows: rhs = [rho (A_fc^T b_fc + A_obs^T b_obs) ; b_eq]."""
    nvn = M.n * M.nv
    g = np.stack([M.rho * (M.A_fc.T @ bfc[ax] + M.A_obs.T @ bobs[ax]) for ax in range(3)])
    rhs = np.concatenate([g, beq], axis=1)
    return (M.Kinv @ rhs.T).T[:, :nvn]


def solve_obstacles(M: Matrices, start, goal, obstacles, max_iters: int, tol: float = 0.0,
                    mode: str = "R2", Ms: list | None = None, stage_iters: int = 1,
                    history: list | None = None):
    """Algorithm 1 with static obstacles (reading R-obst); returns (State of
    the pairs, ObstacleState).  r_max is over pair and obstacle rows.  `Ms`
    (optional): matrices of the rho stages (same n_obs), used as in
    `solve_schedule`."""
    beq = boundary_values(start, goal, M.bc_mask)
    C, a_o, b_o = obstacle_rows(M, obstacles)
    xi = initial_trajectories(M, beq)
    D = pair_differences(M, xi)
    lam = np.zeros_like(D)
    alpha, beta, d, U = projection(D, lam, M, mode)
    Do = obstacle_differences(M, xi, C)
    lam_o = np.zeros_like(Do)
    al_o, be_o, d_o, U_o = projection(Do, lam_o, M, mode, a_o, b_o)
    r = max(residual_max(D - d * U), residual_max(Do - d_o * U_o))
    k = 0
    while k < max_iters:
        Mk = M if Ms is None else Ms[rho_stage(k + 1, len(Ms), stage_iters)]
        bfc = target_vector(alpha, beta, d, lam, Mk)
        bobs = C + target_vector(al_o, be_o, d_o, lam_o, Mk, a_o, b_o)
        xi = qp_step_obstacles(Mk, bfc, bobs, beq)
        D = pair_differences(Mk, xi)
        alpha, beta, d, U = projection(D, lam, Mk, mode)
        lam, fc = lambda_update(lam, D, d, U, Mk.rho)
        Do = obstacle_differences(Mk, xi, C)
        al_o, be_o, d_o, U_o = projection(Do, lam_o, Mk, mode, a_o, b_o)
        lam_o, fco = lambda_update(lam_o, Do, d_o, U_o, Mk.rho)
        r = max(residual_max(fc), residual_max(fco))
        k += 1
        if history is not None:
            history.append(r)
        if r < tol:
            break
    return (State(xi, lam, alpha, beta, d, r, k), ObstacleState(lam_o, al_o, be_o, d_o, r))
