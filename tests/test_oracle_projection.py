"""Pins of the oracle's alpha/beta, d and lambda steps (Eqs. step_alpha,
sphere_project, step_d, lag_update).

* sphere case (l_xy = l_z): the closed form is the exact minimiser of the
  step-alpha objective, checked against a brute-force (alpha, beta) grid;
* spheroid: when the previous d equals the scaled norm of Delta, the closed
  form reaches objective 0;
* the d step is an exact 1-D convex QP: checked against a dense grid;
* the angle form equals the radial form u = Delta / s, s the scaled norm
  (the identity the GPU path relies on), including the degenerate Delta = 0;
* invariants d >= 1, beta in [0, pi], alpha in [-pi, pi].
"""
import numpy as np
import pytest

import oracle as O


class _M:   # the few fields the projection needs
    def __init__(self, a, b, rho=1.0):
        self.a, self.b, self.rho = a, b, rho


def _alpha_objective(D, lam, d_old, al, be, a, b, rho):
    """Objective of Eq. (step_alpha) in the reading of Eq. (sphere_proposed):
    sum over axes of (Delta - d_old * u(alpha, beta) + lambda/rho)^2."""
    U = O.spheroid_direction(al, be, a, b)
    return np.sum((D[:, None] - d_old * U + lam[:, None] / rho) ** 2, axis=0)


@pytest.mark.parametrize("seed", range(6))
def test_sphere_case_closed_form_is_grid_minimiser(seed):
    rng = np.random.default_rng(seed)
    a = b = 0.8
    D = rng.standard_normal(3) * 1.5
    d_old = rng.uniform(1.0, 3.0)
    lam = np.zeros(3)
    al, be = O.alpha_beta(D[:, None], a, b)
    f_closed = _alpha_objective(D, lam, d_old, al, be, a, b, 1.0)[0]
    ga = np.linspace(-np.pi, np.pi, 721)
    gb = np.linspace(0, np.pi, 361)
    AA, BB = np.meshgrid(ga, gb)
    f_grid = _alpha_objective(D, lam, d_old, AA.ravel(), BB.ravel(), a, b, 1.0)
    # closed form is at least as good as every grid point (up to grid step)
    assert f_closed <= f_grid.min() + 1e-12
    # and the grid minimiser lies within one grid step of it on the sphere
    k = np.argmin(f_grid)
    u_grid = O.spheroid_direction(AA.ravel()[k], BB.ravel()[k], a, b)
    u_cl = O.spheroid_direction(al, be, a, b)[:, 0]
    assert np.linalg.norm(u_grid - u_cl) < a * 2 * np.pi / 360 * 1.5


@pytest.mark.parametrize("seed", range(6))
def test_spheroid_closed_form_exact_when_d_matches(seed):
    rng = np.random.default_rng(100 + seed)
    a, b = 0.6, 1.2
    D = rng.standard_normal(3) * 2.0
    s = np.sqrt((D[0] ** 2 + D[1] ** 2) / a ** 2 + D[2] ** 2 / b ** 2)
    al, be = O.alpha_beta(D[:, None], a, b)
    f = _alpha_objective(D, np.zeros(3), s, al, be, a, b, 1.0)[0]
    assert f < 1e-24 * max(1.0, D @ D)


@pytest.mark.parametrize("seed", range(8))
def test_d_step_matches_dense_grid(seed):
    rng = np.random.default_rng(200 + seed)
    W = rng.standard_normal(3) * 2.5
    U = O.spheroid_direction(rng.uniform(-np.pi, np.pi, 1), rng.uniform(0, np.pi, 1), 0.6, 1.2)[:, 0]
    d = O.d_step(W[:, None], U[:, None])[0]
    grid = np.arange(1.0, 10.0, 1e-5)
    f = np.sum((W[:, None] - grid[None] * U[:, None]) ** 2, axis=0)
    f_d = np.sum((W - d * U) ** 2)
    assert f_d <= f.min() + 1e-12
    assert abs(d - grid[np.argmin(f)]) <= 1e-5 or d > 10.0


def test_angle_form_equals_radial_form_and_invariants():
    rng = np.random.default_rng(11)
    a, b = 0.6, 1.2
    D = rng.standard_normal((3, 5000)) * rng.uniform(0.01, 4, 5000)
    # special directions: axes, xy-plane, negative z, tiny and zero vectors
    extra = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 1.0, 0], [0, -2.0, 0], [1.0, 0, 0],
                      [-1.0, 0, 0], [0, 0, 0], [1e-30, 0, 0], [0, 0, -1e-20]]).T
    D = np.concatenate([D, extra], axis=1)
    lam = rng.standard_normal(D.shape) * 0.3
    M = _M(a, b)
    al, be, d, U = O.projection(D, lam, M, "R2")
    assert np.all(d >= 1.0)
    assert np.all((be >= 0) & (be <= np.pi))
    assert np.all((al >= -np.pi) & (al <= np.pi))
    s = np.sqrt((D[0] ** 2 + D[1] ** 2) / a ** 2 + D[2] ** 2 / b ** 2)
    nz = s > 0
    U_rad = np.where(nz, D / np.where(nz, s, 1.0), np.array([[0.0], [0.0], [b]]))
    np.testing.assert_allclose(U, U_rad, atol=1e-13)
    # degenerate Delta = 0 -> alpha = beta = 0 -> u = (0, 0, l_z)
    k0 = D.shape[1] - 3
    assert al[k0] == 0.0 and be[k0] == 0.0
    # R3: d = max(1, s) exactly in the radial form
    _, _, d3, _ = O.projection(D, lam, M, "R3")
    np.testing.assert_allclose(d3[nz], np.maximum(1.0, s[nz]), rtol=1e-13)


def test_lambda_update_and_target():
    rng = np.random.default_rng(3)
    M = _M(0.6, 1.2, rho=2.0)
    D = rng.standard_normal((3, 50))
    lam = rng.standard_normal((3, 50))
    al, be, d, U = O.projection(D, lam, M, "R2")
    lam2, fc = O.lambda_update(lam, D, d, U, M.rho)
    np.testing.assert_allclose(fc, D - d * U)
    np.testing.assert_allclose(lam2, lam + 2.0 * fc)
    bfc = O.target_vector(al, be, d, lam2, M)
    np.testing.assert_allclose(bfc, d * U - lam2 / 2.0)
    # a pair-time outside the scaled spheroid with lambda = 0 has f_c = 0 (R3)
    Dfar = np.array([[3.0], [0.0], [0.0]])
    _, _, dfar, Ufar = O.projection(Dfar, np.zeros((3, 1)), M, "R3")
    assert np.abs(Dfar - dfar * Ufar).max() < 1e-15
