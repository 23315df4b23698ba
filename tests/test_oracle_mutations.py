"""Mutation checks of the oracle's pins.

Each case plants a plausible mistake into the oracle (on the CPU, by
monkeypatching one function) and checks that at least one pin test fails.
This shows the pins are strong enough to catch a dropped term, a wrong
sign or index, or a swapped operand.
"""
import numpy as np
import pytest

import oracle
import oracle.amto_oracle as OA
import tests.test_oracle_basis as TB
import tests.test_oracle_convergence as TC
import tests.test_oracle_kkt as TK
import tests.test_oracle_projection as TP
import tests.test_oracle_obstacles as TO
import tests.test_oracle_planar as TPL
import tests.test_oracle_qp as TQ
import tests.test_oracle_residual as TR


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _pair_matrix_signs_swapped(P, n):
    return -_orig["pair_matrix"](P, n)


def _lambda_update_wrong_sign(lam, D, d, U, rho):
    fc = D - d * U
    return lam - rho * fc, fc


def _target_without_lambda(alpha, beta, d, lam, M):
    return d * OA.spheroid_direction(alpha, beta, M.a, M.b)


def _alpha_beta_axes_swapped(D, a, b):
    return _orig["alpha_beta"](D, b, a)


def _d_step_unclipped(W, U):
    return np.sum(W * U, axis=0) / np.sum(U * U, axis=0)


def _boundary_rows_off_by_one(P, dP, ddP, bc_mask=OA.BC_ALL):
    rows = [P[1], dP[0], ddP[0], P[-1], dP[-1], ddP[-1]]
    return np.stack([r for i, r in enumerate(rows) if (bc_mask >> i) & 1])


def _qp_step_without_rho(M, bfc, beq):
    nvn = M.n * M.nv
    rhs = np.concatenate([np.stack([M.A_fc.T @ bfc[ax] for ax in range(3)]), beq], axis=1)
    return (M.Kinv @ rhs.T).T[:, :nvn]


def _basis_derivative_sign(degree, m, T):
    P, dP, ddP = _orig["bernstein_basis"](degree, m, T)
    return P, -dP, ddP


def _obstacle_difference_sign(M, xi, C):
    return C - np.stack([M.A_obs @ xi[ax] for ax in range(3)])


def _obstacle_axes_swapped(M, obstacles):
    C, a_o, b_o = _orig["obstacle_rows"](M, obstacles)
    return C, b_o, a_o


def _obstacle_rows_missing_from_gram(P, n, n_obs):
    return _orig["obstacle_matrix"](P, n, 0)


def _planar_angle_axes_swapped(D, lam, M, mode="R2", a=None, b=None):
    if not getattr(M, "planar", False):
        return _orig["projection"](D, lam, M, mode, a, b)
    a = M.a if a is None else a
    alpha = np.arctan2(D[0], D[1])
    U = np.stack([a * np.cos(alpha), a * np.sin(alpha), np.zeros_like(alpha)])
    Wd = D if mode == "R3" else D + lam / M.rho
    return alpha, np.full_like(alpha, np.pi / 2), OA.d_step(Wd, U), U


def _residual_inf_norm(fc):
    return float(np.abs(fc).max()) if fc.size else 0.0


def _residual_rms(fc):
    return float(np.sqrt(np.mean(np.sum(fc * fc, axis=0)))) if fc.size else 0.0


def _residual_squared(fc):
    return float(np.max(np.sum(fc * fc, axis=0))) if fc.size else 0.0


_orig = {k: getattr(OA, k) for k in ["pair_matrix", "alpha_beta", "bernstein_basis",
                                     "obstacle_rows", "obstacle_matrix", "projection"]}

MUTATIONS = {
    "pair signs swapped": ("pair_matrix", _pair_matrix_signs_swapped,
                           [(TQ.test_qp_step_matches_independent_least_squares, 3, 1)]),
    "lambda update sign": ("lambda_update", _lambda_update_wrong_sign,
                           [(TC.test_r3_swap_residual_monotone_to_machine_precision,)]),
    "lambda dropped from b_fc": ("target_vector", _target_without_lambda,
                                 [(TC.test_r3_swap_residual_monotone_to_machine_precision,)]),
    "l_xy and l_z swapped": ("alpha_beta", _alpha_beta_axes_swapped,
                             [(TP.test_spheroid_closed_form_exact_when_d_matches, 0)]),
    "d not clipped": ("d_step", _d_step_unclipped,
                      [(TP.test_angle_form_equals_radial_form_and_invariants,)]),
    "wrong boundary row": ("boundary_rows", _boundary_rows_off_by_one,
                           [(TB.test_boundary_rows_select_by_mask,),
                            (TQ.test_initial_trajectories_are_straight_segments,)]),
    "rho dropped from rhs": ("qp_step", _qp_step_without_rho,
                             [(TQ.test_qp_step_kkt_optimality_and_boundary_exactness,)]),
    "derivative sign": ("bernstein_basis", _basis_derivative_sign,
                        [(TB.test_derivatives_match_symbolic_differentiation, 10, 50, 5.0)]),
    "obstacle difference sign": ("obstacle_differences", _obstacle_difference_sign,
                                 [(TO.test_solutions_clear_the_obstacle, "R3")]),
    "obstacle l_xy and l_z swapped": ("obstacle_rows", _obstacle_axes_swapped,
                                      [(TO.test_single_detour_touches_the_obstacle, "R3", 1.2)]),
    "obstacle rows missing": ("obstacle_matrix", _obstacle_rows_missing_from_gram,
                              [(TO.test_gram_and_inverse_closed_forms, 3, 1, 1.0)]),
    "residual as largest component": ("residual_max", _residual_inf_norm,
                                      [(TR.test_residual_max_is_largest_column_euclidean_norm,),
                                       (TR.test_residual_of_crossing_pair_closed_form, 0.2)]),
    "residual as RMS": ("residual_max", _residual_rms,
                        [(TR.test_residual_max_is_largest_column_euclidean_norm,),
                         (TR.test_residual_of_crossing_pair_closed_form, 0.2)]),
    "residual squared (no root)": ("residual_max", _residual_squared,
                                   [(TR.test_residual_of_crossing_pair_closed_form, 0.2)]),
    "planar angle axes swapped": ("projection", _planar_angle_axes_swapped,
                                  [(TPL.test_lambda_free_residual_inside_the_disk,)]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn, checks = MUTATIONS[name]
    monkeypatch.setattr(OA, attr, fn)        # calls inside the oracle
    monkeypatch.setattr(oracle, attr, fn)    # calls through the package
    caught = [_fails(c[0], *c[1:]) for c in checks]
    assert any(caught), f"mutation '{name}' was not caught by its pins"


def test_unmutated_pins_pass():
    for _, _, checks in MUTATIONS.values():
        for c in checks:
            c[0](*c[1:])
