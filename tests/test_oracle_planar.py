"""Pins of the oracle's planar (2-D disk) reading R-planar (Sec. III: agents
modelled as disks in 2D).

* away from exact coincidences the planar solve is the 3-D solve of the same
  in-plane problem (for Delta_z = 0 the spheroid projection has beta = pi/2);
* Delta = 0 projects on +x (alpha = atan2(0, 0) = 0), not on the 3-D +z;
* the lambda-free residual of a pair inside the disk is Delta (1 - l/|Delta|);
* in-plane swaps whose straight paths meet at the centre, and random planar
  boxes, separate every pair to the disk radius and keep z at exactly 0.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _planar_problem(n, seed, m=40, T=5.0):
    prob = W.random_box(n, seed, box=(6.0, 6.0, 0.0), m=m, T=T)
    s, g = O.planar_inputs(prob.start, prob.goal)
    return prob, s, g


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_planar_equals_3d_in_the_plane(mode):
    prob, s, g = _planar_problem(6, 3)
    Mp = O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho,
                          planar=True)
    M3 = O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho)
    sp_ = O.solve(Mp, s, g, 30, mode=mode)
    s3 = O.solve(M3, s, g, 30, mode=mode)
    np.testing.assert_allclose(sp_.xi[:2], s3.xi[:2], rtol=0, atol=1e-10 * np.abs(s3.xi).max())
    assert np.all(sp_.xi[2] == 0.0)
    assert abs(sp_.r_max - s3.r_max) < 1e-10


def test_coincident_agents_project_on_plus_x():
    Mp = O.build_matrices(2, 20, 10, 3.0, 0.6, 1.2, 1.0, planar=True)
    D = np.zeros((3, 5))
    alpha, beta, d, U = O.projection(D, np.zeros_like(D), Mp, "R2")
    np.testing.assert_array_equal(alpha, 0.0)
    np.testing.assert_allclose(U, np.array([[0.6] * 5, [0.0] * 5, [0.0] * 5]))
    np.testing.assert_array_equal(d, 1.0)


def test_lambda_free_residual_inside_the_disk():
    Mp = O.build_matrices(2, 20, 10, 3.0, 0.6, 1.2, 1.0, planar=True)
    rng = np.random.default_rng(4)
    ang = rng.uniform(-np.pi, np.pi, 50)
    rad = rng.uniform(0.05, 1.5, 50)
    D = np.stack([rad * np.cos(ang), rad * np.sin(ang), np.zeros(50)])
    _, _, d, U = O.projection(D, np.zeros_like(D), Mp, "R3")
    f = D - d * U
    ref = D * np.minimum(0.0, 1.0 - 0.6 / rad)
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-14)


def _circle_swap_plane(n=4, m=41):
    th = 2 * np.pi * np.arange(n) / n
    start = np.stack([2.5 * np.cos(th), 2.5 * np.sin(th), np.zeros(n)], 1).astype(np.float32)
    goal = start.copy()
    goal[:, :2] *= -1
    return W.Problem(n=n, m=m, T=5.0, start=start, goal=goal)


@pytest.mark.parametrize("mode,n", [("R3", 4), ("R3", 5)])
def test_centre_crossing_swap_separates_in_plane(mode, n):
    """(On these symmetric swaps the literal reading depends on the rounding
    left where all paths meet and does not settle; it is checked on random
    planar boxes below.)"""
    prob = _circle_swap_plane(n)
    Mp = O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho,
                          planar=True)
    s, g = O.planar_inputs(prob.start, prob.goal)
    st0 = O.init_state(Mp, O.boundary_values(s, g), mode)
    assert np.abs(O.pair_differences(Mp, st0.xi)).sum(axis=0).min() < 1e-12  # they meet
    st = O.solve(Mp, s, g, 2000, 1e-4, mode=mode)
    assert st.r_max < 1e-4
    assert np.all(st.xi[2] == 0.0)
    pos = O.positions(Mp, st.xi)
    for i in range(prob.n):
        for j in range(i + 1, prob.n):
            assert np.hypot(*(pos[:2, i] - pos[:2, j])).min() > prob.a * (1 - 1e-3)


@pytest.mark.parametrize("seed", [1, 2])
def test_random_planar_box_separates(seed):
    prob = W.random_box(6, seed, box=(6.0, 6.0, 0.0), m=40, T=5.0)
    Mp = O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho,
                          planar=True)
    s, g = O.planar_inputs(prob.start, prob.goal)
    st = O.solve(Mp, s, g, 2000, 1e-4, mode="R2")
    assert st.r_max < 1e-4
    assert np.all(st.xi[2] == 0.0)
    pos = O.positions(Mp, st.xi)
    for i in range(prob.n):
        for j in range(i + 1, prob.n):
            assert np.hypot(*(pos[:2, i] - pos[:2, j])).min() > prob.a * (1 - 1e-3)
