"""Pins of the oracle's residual norm (Algorithm 1's stopping test, reading
R-stop: the largest Euclidean norm of f_c over all pairs and samples).

Two independent fixes:
  * hand-built f_c columns whose largest 2-norm differs from their largest
    component, their RMS and their largest column sum;
  * a closed form: two agents whose straight initial trajectories (reading
    R-init) cross with a closest approach delta along a diagonal of the x-y
    plane.  In the lambda-free reading f_c = Delta min(0, 1 - 1/s), so at the
    closest approach ||f_c|| = l_xy - delta, while its largest component is
    0.8 (l_xy - delta).
"""
import numpy as np
import pytest

import oracle.amto_oracle as OA


def test_residual_max_is_largest_column_euclidean_norm():
    # columns (3, 4, 0) and (0, 0, 4.5): 2-norms 5 and 4.5; largest component
    # 4.5; RMS over the columns sqrt((25 + 20.25) / 2); largest |.| sum 7
    fc = np.array([[3.0, 0.0], [4.0, 0.0], [0.0, 4.5]])
    assert OA.residual_max(fc) == pytest.approx(5.0, abs=1e-15)
    # order of the columns and a zero column do not matter
    fc2 = np.concatenate([np.zeros((3, 1)), fc[:, ::-1]], axis=1)
    assert OA.residual_max(fc2) == pytest.approx(5.0, abs=1e-15)
    # single column along an axis: the norm is the magnitude of the entry
    assert OA.residual_max(np.array([[0.0], [-2.5], [0.0]])) == pytest.approx(2.5, abs=1e-15)
    # no pairs (one agent): no constraint, residual 0
    assert OA.residual_max(np.zeros((3, 0))) == 0.0


@pytest.mark.parametrize("delta", [0.1, 0.2, 0.45])
def test_residual_of_crossing_pair_closed_form(delta):
    a, b = 0.6, 1.2
    M = OA.build_matrices(2, 51, 10, 5.0, a, b, 1.0)
    v = np.array([0.8, -0.6, 0.0])   # relative motion
    w = np.array([0.6, 0.8, 0.0])    # closest-approach direction, v . w = 0
    c = np.array([0.0, 0.0, 1.0])
    d0, d1 = -4.0 * v + delta * w, 4.0 * v + delta * w   # Delta at t = 0 and t = T
    start = np.stack([c + d0 / 2, c - d0 / 2])
    goal = np.stack([c + d1 / 2, c - d1 / 2])
    beq = OA.boundary_values(start, goal, M.bc_mask)
    st = OA.init_state(M, beq, mode="R3")
    # rest-to-rest profile is symmetric: sample 25 (t = T/2) is the midpoint,
    # where Delta = delta w; ||f_c|| = |Delta| (1/s - 1) = l_xy - delta there
    # and smaller at every other sample
    assert st.r_max == pytest.approx(a - delta, abs=1e-9)
    D = OA.pair_differences(M, st.xi)
    np.testing.assert_allclose(D[:, 25], delta * w, atol=1e-9)
