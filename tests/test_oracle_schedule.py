"""Pins of the increasing-rho schedule (Sec. IV-A; reading R-rho-sched).

The schedule only changes which penalty (and cached inverse) an iteration
uses.  Pinned: a constant schedule is the plain solve; the stage function;
at a stage switch the QP step is the minimiser of the stage's own objective
(independent null-space least-squares solve with that rho); and the paper's
motivation, that increasing rho reaches the residual tolerance in fewer
iterations on the same problem."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.test_oracle_qp import _independent_qp


def _mats(prob, rho):
    return O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, rho)


def test_stage_function():
    assert [O.rho_stage(k, 3, 4) for k in range(1, 15)] == [0] * 4 + [1] * 4 + [2] * 6
    assert [O.rho_stage(k, 1, 5) for k in range(1, 8)] == [0] * 7


def test_constant_schedule_is_the_plain_solve():
    prob = W.random_box(6, 3, box=(6.0, 6.0, 3.0), m=30, T=4.0)
    M = _mats(prob, 1.0)
    ref = O.solve(M, prob.start, prob.goal, 25)
    st = O.solve_schedule([M, M, M], 7, prob.start, prob.goal, 25)
    assert np.array_equal(st.xi, ref.xi) and np.array_equal(st.lam, ref.lam)
    assert st.r_max == ref.r_max and st.k == ref.k


@pytest.mark.parametrize("mode", ["R2", "R3"])
def test_switch_iteration_solves_the_new_stage_qp(mode):
    """Iteration E+1 is the first of stage 1: its QP uses rho_1 = g rho_0 with the
    multipliers carried over, b = S - lambda / rho_1 (Eq. b_f)."""
    prob = W.random_box(3, 5, box=(4.0, 4.0, 2.0), m=20, T=4.0)
    Ms = [_mats(prob, 1.0), _mats(prob, 3.0)]
    E = 4
    before = O.solve_schedule(Ms, E, prob.start, prob.goal, E, mode=mode)
    after = O.solve_schedule(Ms, E, prob.start, prob.goal, E + 1, mode=mode)
    M1 = Ms[1]
    bfc = O.target_vector(before.alpha, before.beta, before.d, before.lam, M1)
    beq = O.boundary_values(prob.start, prob.goal)
    for ax in range(3):
        ref = _independent_qp(M1.P, M1.ddP, M1.A, prob.n, 3.0, bfc[ax], beq[ax])
        np.testing.assert_allclose(after.xi[ax], ref, rtol=0, atol=1e-8 * np.abs(ref).max())
    # the multipliers of iteration E+1 are updated with rho_1
    D = O.pair_differences(M1, after.xi)
    _, _, d, U = O.projection(D, before.lam, M1, mode=mode)
    lam, _ = O.lambda_update(before.lam, D, d, U, 3.0)
    np.testing.assert_allclose(after.lam, lam, rtol=0, atol=1e-12)


def test_increasing_rho_reaches_the_tolerance_sooner():
    """Sec. IV-A: the larger penalties of the later iterations speed up the
    loop; 16 agents in a 6x6x3 m box, tol 1e-2."""
    prob = W.box16(0)
    hist = []
    plain = O.solve(_mats(prob, 1.0), prob.start, prob.goal, 300, 1e-2)
    g = 100 ** (1 / 9)
    Ms = [_mats(prob, g ** j) for j in range(10)]
    sched = O.solve_schedule(Ms, 10, prob.start, prob.goal, 300, 1e-2, history=hist)
    assert plain.r_max < 1e-2 and sched.r_max < 1e-2
    assert sched.k < 0.75 * plain.k, (sched.k, plain.k)
