"""Static obstacles on the GPU (Sec. IV-A; reading R-obst).

Each (agent, obstacle, sample) is a pair row with a fixed partner, processed
by the pair kernel after the agent pairs of each time block (its multipliers
continue the same stream); the KKT inverse carries n_obs rho P^T P per agent.
Checked against the oracle's `solve_obstacles` in both readings, both
multiplier forms, the tensor-core and structured applies and the rho
schedule; solutions clear the obstacles; the reported residual is the FP64
maximum over pair and obstacle rows; bad obstacle data and missing obstacles
are rejected.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import rel_inf, to_dev

pytestmark = pytest.mark.gpu
MODES = {"R2": 0, "R3": 1}
MULT = {"auto": 0, "pairs": 1, "aggregate": 2}
XI_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _planner(prob, n_obs, B=1, mode="R2", mult="auto", apply_mode=0, precision=0, **kw):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree,
                   proj_mode=MODES[mode], max_batch=B, apply_mode=apply_mode,
                   precision=precision, multipliers=MULT[mult], n_obstacles=n_obs, **kw)


def _solve(pl, probs, obsts, iters, tol=0.0):
    import torch
    s, g = W.stack(probs)
    dev = pl.device
    pl.set_obstacles(to_dev(np.stack(obsts), dev))
    xi, r, k = pl.solve(to_dev(s, dev), to_dev(g, dev), iters, tol)
    torch.cuda.synchronize()
    return xi.cpu().numpy(), r.cpu().numpy(), k.cpu().numpy()


def _oracle(prob, obst, k, mode, tol=0.0, rho_sched=None):
    n_obs = obst.shape[0]
    mk = lambda rho: O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b,  # noqa
                                      rho, n_obs=n_obs)
    if rho_sched:
        J, g, E = rho_sched
        Ms = [mk(prob.rho * g ** j) for j in range(J)]
        return O.solve_obstacles(Ms[0], prob.start, prob.goal, obst, k, tol, mode, Ms=Ms,
                                 stage_iters=E)
    return O.solve_obstacles(mk(prob.rho), prob.start, prob.goal, obst, k, tol, mode)


@pytest.mark.parametrize("n,n_obs,mode,mult,k", [
    (4, 1, "R2", "auto", 5), (16, 3, "R2", "auto", 20), (16, 8, "R3", "aggregate", 30),
    (16, 8, "R3", "pairs", 30), (33, 5, "R2", "auto", 10), (24, 2, "R3", "aggregate", 40),
    (9, 4, "R2", "auto", 1), (64, 6, "R3", "aggregate", 3)])
def test_matches_oracle(n, n_obs, mode, mult, k):
    box = (10.0, 10.0, 5.0) if n == 64 else (7.0, 7.0, 3.5)
    prob, obst = W.obstacle_box(n, n_obs, 100 + n + n_obs, box=box, m=60, T=6.0)
    pl = _planner(prob, n_obs, mode=mode, mult=mult, loop_mode=1)
    assert pl.info.n_obstacles == n_obs
    x, r, kk = _solve(pl, [prob], [obst], k)
    assert kk[0] == k
    st, _ = _oracle(prob, obst, k, mode)
    assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, rel_inf(x[0].reshape(3, -1), st.xi)
    assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2), (r[0], st.r_max)


@pytest.mark.parametrize("precision,apply_mode,tol", [(1, 0, 1e-4), (0, 3, 1e-4), (2, 0, 1e-3)])
def test_batched_applies(precision, apply_mode, tol):
    """A batch with different obstacles per instance through the tensor-core
    (TF32X3, BF16X3) and the structured apply."""
    B, n, n_obs, k = 5, 16, 4, 15
    pairs = [W.obstacle_box(n, n_obs, 300 + i, box=(7.0, 7.0, 3.5), m=50, T=6.0)
             for i in range(B)]
    probs, obsts = [p for p, _ in pairs], [o for _, o in pairs]
    pl = _planner(probs[0], n_obs, B=B, precision=precision, apply_mode=apply_mode, loop_mode=1)
    x, r, kk = _solve(pl, probs, obsts, k)
    for i in (0, B - 1):
        st, _ = _oracle(probs[i], obsts[i], k, "R2")
        assert rel_inf(x[i].reshape(3, -1), st.xi) < tol


def test_rho_schedule_with_obstacles():
    prob, obst = W.obstacle_box(12, 3, 7, box=(6.0, 6.0, 3.0), m=50, T=6.0)
    J, g, E = 3, 3.0, 4
    pl = _planner(prob, 3, mode="R2", loop_mode=1, rho_stages=J, rho_growth=g,
                  rho_stage_iters=E)
    for k in (E + 1, 2 * E + 2):
        x, r, kk = _solve(pl, [prob], [obst], k)
        st, _ = _oracle(prob, obst, k, "R2", rho_sched=(J, g, E))
        assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, k


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_solutions_clear_the_obstacle(mode):
    """The oracle's crossing scene to tolerance on the GPU: every agent clears
    the obstacle.  (The scene is four-fold symmetric, so float32 and FP64
    iterates part after a few iterations and their iteration counts to the
    tolerance differ; they are compared on the detour scene below.)"""
    start = np.array([[-3.0, 0.2, 1.0], [3.0, -0.2, 1.0], [0.2, -3.0, 1.0], [-0.2, 3.0, 1.0]],
                     np.float32)
    goal = np.array([[3.0, -0.2, 1.0], [-3.0, 0.2, 1.0], [-0.2, 3.0, 1.0], [0.2, -3.0, 1.0]],
                    np.float32)
    obst = np.array([[0.05, 0.1, 1.0, 1.0, 1.4]], np.float32)
    prob = W.Problem(n=4, m=60, T=6.0, start=start, goal=goal)
    pl = _planner(prob, 1, mode=mode, loop_mode=1)
    x, r, kk = _solve(pl, [prob], [obst], 1500, 2e-3)
    assert r[0] < 2e-3 * 1.001 and kk[0] < 1500
    M = O.build_matrices(4, 60, prob.degree, 6.0, prob.a, prob.b, prob.rho, n_obs=1)
    pos = O.positions(M, x[0].reshape(3, -1).astype(np.float64))
    d = pos - obst[0, :3, None, None].astype(np.float64)
    s = np.sqrt((d[0] ** 2 + d[1] ** 2) / 1.0 ** 2 + d[2] ** 2 / 1.4 ** 2)
    assert s.min() > 1.0 - 5e-3


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_detour_to_tolerance_matches_oracle(mode):
    """One agent detours around an obstacle on its straight path: iteration
    count to the tolerance and the trajectories agree with the oracle."""
    start = np.array([[-3.0, 0.2, 1.0], [-3.0, 2.8, 1.0]], np.float32)
    goal = np.array([[3.0, 0.2, 1.0], [3.0, 2.8, 1.0]], np.float32)
    obst = np.array([[0.0, 0.0, 1.0, 1.0, 1.4]], np.float32)
    prob = W.Problem(n=2, m=60, T=6.0, start=start, goal=goal)
    pl = _planner(prob, 1, mode=mode, loop_mode=1)
    x, r, kk = _solve(pl, [prob], [obst], 1500, 1e-3)
    st, _ = _oracle(prob, obst, 1500, mode, tol=1e-3)
    assert abs(int(kk[0]) - st.k) <= max(2, 0.02 * st.k), (kk[0], st.k)
    if int(kk[0]) == st.k:
        assert rel_inf(x[0].reshape(3, -1), st.xi) < 1e-3


@pytest.mark.parametrize("mult", ["aggregate", "pairs"])
def test_reported_residual_is_the_fp64_maximum(mult):
    """Recompute every pair and obstacle residual of the lambda-free reading in
    FP64 from the returned coefficients: the maximum is the reported one."""
    B, n, n_obs = 3, 16, 6
    pairs = [W.obstacle_box(n, n_obs, 500 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0)
             for i in range(B)]
    probs, obsts = [p for p, _ in pairs], [o for _, o in pairs]
    pl = _planner(probs[0], n_obs, B=B, mode="R3", mult=mult, loop_mode=1)
    x, r, kk = _solve(pl, probs, obsts, 4)
    M = O.build_matrices(n, 50, probs[0].degree, 6.0, probs[0].a, probs[0].b, probs[0].rho,
                         n_obs=n_obs)
    for i in range(B):
        xi = x[i].reshape(3, -1).astype(np.float64)
        D = O.pair_differences(M, xi)
        _, _, dd, U = O.projection(D, np.zeros_like(D), M, "R3")
        C, ao, bo = O.obstacle_rows(M, obsts[i].astype(np.float64))
        Do = O.obstacle_differences(M, xi, C)
        _, _, do, Uo = O.projection(Do, np.zeros_like(Do), M, "R3", ao, bo)
        ref = max(O.residual_max(D - dd * U), O.residual_max(Do - do * Uo))
        assert abs(r[i] - ref) <= 1e-5 * max(ref, 1e-3), (i, r[i], ref)


def test_rejections_and_bad_obstacles():
    from paper_2011_04240_b300 import amto
    prob, obst = W.obstacle_box(8, 2, 9, box=(6.0, 6.0, 3.0), m=40, T=5.0)
    pl = _planner(prob, 2, B=2, loop_mode=1)
    s, g = W.stack([prob, prob])
    with pytest.raises(amto.AmtoError):  # obstacles not set
        pl.solve(to_dev(s, pl.device), to_dev(g, pl.device), 5)
    bad = np.stack([obst, obst]).copy()
    bad[1, 0, 3] = -1.0  # a negative semi-axis
    pl.set_obstacles(to_dev(bad, pl.device))
    import torch
    xi, r, k = pl.solve(to_dev(s, pl.device), to_dev(g, pl.device), 5)
    torch.cuda.synchronize()
    assert int(k[0]) == 5 and int(k[1]) == -1 and np.isnan(float(r[1]))
    # plans without obstacles reject amto_set_obstacles; plans with them the
    # block solver and mixed batches
    p0 = _planner(prob, 0)
    ob_dev = to_dev(np.stack([obst]), p0.device)
    assert amto.load().amto_set_obstacles(p0.plan, 1, ob_dev.data_ptr(), None) == amto.EINVAL
    with pytest.raises(amto.AmtoError):
        _planner(prob, 2, loop_mode=2)
    assert _planner(prob, 2).info.loop_mode == amto.LOOP_GRAPH  # automatic loop yields
    from paper_2011_04240_b300 import Mixed
    with pytest.raises(amto.AmtoError):
        Mixed([pl])
