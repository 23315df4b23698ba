"""Planar plans (disks in the x-y plane; Sec. III "disks in 2D", reading
R-planar) on the GPU.

The library runs the disk problem through its spheroid kernels with the axes
permuted (the plane's x on the kernels' z, so that Delta = 0 projects on the
plane's +x) and l_z = l_xy.  Checked against the oracle's planar reading:
random planar boxes in both readings and multiplier forms, exactly
coincident agents (Delta = 0 at every sample), obstacles, warm starts, the
block solver and the state read-back; every z input is ignored and every z
output is 0.
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


def _planner(prob, B=1, mode="R2", mult="auto", **kw):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, 99.0, prob.rho, prob.degree,
                   proj_mode=MODES[mode], max_batch=B, multipliers=MULT[mult], planar=1, **kw)


def _mats(prob, n_obs=0):
    return O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho,
                            n_obs=n_obs, planar=True)


def _gpu(pl, probs, k, tol=0.0, **kw):
    """Solve with random z in every input (ignored by planar plans)."""
    import torch
    s, g = W.stack(probs)
    rng = np.random.default_rng(0)
    s = s.copy()
    g = g.copy()
    s[..., 2] = rng.uniform(-5, 5, s.shape[:-1])
    g[..., 2] = rng.uniform(-5, 5, g.shape[:-1])
    dev = pl.device
    xi, r, kk = pl.solve(to_dev(s, dev), to_dev(g, dev), k, tol,
                         **{key: to_dev(v, dev) for key, v in kw.items()})
    torch.cuda.synchronize()
    return xi.cpu().numpy(), r.cpu().numpy(), kk.cpu().numpy()


def _box(n, seed, m=50):
    side = 6.0 if n <= 16 else 9.0
    prob = W.random_box(n, seed, box=(side, side, 0.0), m=m, T=5.0)
    return prob


def _oracle(prob, k, mode, tol=0.0, obst=None):
    s, g = O.planar_inputs(prob.start, prob.goal)
    if obst is None:
        return O.solve(_mats(prob), s, g, k, tol, mode)
    ob = np.array(obst, np.float64)
    ob[:, 2] = 0.0
    st, _ = O.solve_obstacles(_mats(prob, ob.shape[0]), s, g, ob, k, tol, mode)
    return st


@pytest.mark.parametrize("n,mode,mult,k,loop", [
    (3, "R2", "auto", 10, 0), (8, "R2", "auto", 30, 2), (16, "R2", "auto", 40, 1),
    (16, "R3", "aggregate", 40, 1), (16, "R3", "pairs", 40, 1), (33, "R2", "auto", 15, 1)])
def test_matches_planar_oracle(n, mode, mult, k, loop):
    prob = _box(n, 20 + n)
    pl = _planner(prob, mode=mode, mult=mult, loop_mode=loop)
    assert pl.info.planar == 1
    x, r, kk = _gpu(pl, [prob], k)
    st = _oracle(prob, k, mode)
    assert kk[0] == k
    assert np.all(x[0, 2] == 0.0)
    assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, rel_inf(x[0].reshape(3, -1), st.xi)
    assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2)


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_coincident_agents_separate_along_x(mode):
    """Two agents with the same start and goal coincide exactly at every sample
    of the initial trajectories (identical arithmetic): their Delta = 0
    projects on the plane's +x (the kernels' degenerate direction, permuted),
    as the oracle's atan2(0, 0) = 0 does."""
    # (the third agent stays well away: a near-coincidence formed by rounding
    # would give the two sides different directions)
    start = np.array([[-2.0, 0.5, 0.0], [-2.0, 0.5, 0.0], [0.5, 3.0, 0.0]], np.float32)
    goal = np.array([[2.0, -0.5, 0.0], [2.0, -0.5, 0.0], [0.0, 4.5, 0.0]], np.float32)
    prob = W.Problem(n=3, m=41, T=5.0, start=start, goal=goal)
    pl = _planner(prob, mode=mode, loop_mode=1)
    for k in (1, 3):
        x, r, kk = _gpu(pl, [prob], k)
        st = _oracle(prob, k, mode)
        assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, (k, rel_inf(x[0].reshape(3, -1), st.xi))
        # the pair moved apart along x (in the plane), not along y
        xa = x[0].reshape(3, 3, -1)
        assert np.abs(xa[0, 0] - xa[0, 1]).max() > 1e-3


def test_planar_obstacles():
    prob, obst = W.obstacle_box(10, 3, 11, box=(6.0, 6.0, 0.0), m=50, T=5.0)
    ob = obst.copy()
    ob[:, 2] = 7.0       # ignored: centres in the plane
    ob[:, 4] = 0.01      # ignored: disks use l_xy
    pl = _planner(prob, mode="R2", loop_mode=1, n_obstacles=3)
    pl.set_obstacles(to_dev(ob[None], pl.device))
    x, r, kk = _gpu(pl, [prob], 20)
    st = _oracle(prob, 20, "R2", obst=obst)
    assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL


@pytest.mark.parametrize("mult", ["pairs", "aggregate"])
def test_planar_warm_start(mult):
    """One iteration from the oracle's planar state after 15 iterations (the
    trajectories and multipliers passed in the plane's axes, z rows noise)."""
    prob = _box(12, 7)
    M = _mats(prob)
    s, g = O.planar_inputs(prob.start, prob.goal)
    st15 = O.solve(M, s, g, 15, mode="R3")
    xi0 = st15.xi.astype(np.float32).reshape(1, 3, 12, -1)
    lam0 = st15.lam.astype(np.float32).reshape(1, 3, 66, prob.m)
    xi0 = xi0.copy()
    lam0 = lam0.copy()
    xi0[:, 2] = 3.0
    lam0[:, 2] = 5.0
    ws = O.warm_state(M, st15.xi, st15.lam, "R3")
    ref = O.am_iteration(M, ws, O.boundary_values(s, g), "R3")
    pl = _planner(prob, mode="R3", mult=mult, loop_mode=1)
    x, r, kk = _gpu(pl, [prob], 1, xi_init=xi0, lambda_init=lam0)
    assert rel_inf(x[0].reshape(3, -1), ref.xi) < XI_TOL


def test_planar_state_read_back():
    import torch
    prob = _box(6, 9)
    pl = _planner(prob, mode="R2", mult="pairs", loop_mode=1)
    x, r, kk = _gpu(pl, [prob], 8)
    lam, al, be, d = pl.state()
    torch.cuda.synchronize()
    lam, al, be, d = (v.cpu().numpy() for v in (lam, al, be, d))
    st = _oracle(prob, 8, "R2")
    floor = max(np.abs(st.lam).max(), 1e-2)
    assert np.abs(lam[0].reshape(3, -1) - st.lam).max() / floor < 1e-4
    assert np.all(lam[0, 2] == 0.0)
    np.testing.assert_allclose(be, np.pi / 2, atol=1e-6)
    D = O.pair_differences(_mats(prob), st.xi)
    big = np.hypot(D[0], D[1]) > 1e-3
    da = np.angle(np.exp(1j * (al[0].ravel() - st.alpha)))
    assert np.abs(da[big]).max() < 1e-3
    np.testing.assert_allclose(d[0].ravel(), st.d, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_sphere_agents(mode):
    """The sphere specialization (l_xy = l_z) of the 3-D spheroid path."""
    from paper_2011_04240_b300 import Planner
    prob = W.random_box(12, 77, box=(6.0, 6.0, 3.0), m=50, T=5.0)
    pl = Planner(prob.n, prob.m, prob.T, 0.8, 0.8, prob.rho, prob.degree,
                 proj_mode=MODES[mode], loop_mode=1)
    s, g = W.stack([prob])
    import torch
    xi, r, kk = pl.solve(to_dev(s, pl.device), to_dev(g, pl.device), 25)
    torch.cuda.synchronize()
    M = O.build_matrices(prob.n, prob.m, prob.degree, prob.T, 0.8, 0.8, prob.rho)
    st = O.solve(M, prob.start, prob.goal, 25, mode=mode)
    assert rel_inf(xi.cpu().numpy()[0].reshape(3, -1), st.xi) < XI_TOL
