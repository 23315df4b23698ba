"""Parity at the benchmark's full size and launch configuration.

The timed workload: 256 instances of the 64-agent antipodal shell (m = 100),
lambda-free projection (reading R3) with aggregated multipliers, TF32X3
cached-inverse apply, one plan of max_batch 256 solving the whole batch from
device-resident inputs.  Outputs the FP64 oracle can compute one by one are
compared on four sampled instances; at the benchmark's 20 iterations, past
the shell's parity horizon (its trajectories are chaotic after a few
iterations, so the float32 and FP64 iterates separate), properties that hold
at any size are checked instead: the boundary conditions (Eq. eq_step_x), the
reported residual being the FP64 maximum of Algorithm 1's stopping norm at
the returned iterate, and an instance's result not depending on the batch it
is solved in.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import gpu_solve, oracle_mats, oracle_solve, planner, rel_inf

pytestmark = pytest.mark.gpu

B, N_AGENTS = 256, 64
SAMPLES = (0, 85, 170, 255)
XI_TOL = 1e-4


@pytest.fixture(scope="module")
def bench_plan():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    probs = W.shell_batch(B, seed=0, n=N_AGENTS)
    pl = planner(probs[0], "R3", max_batch=B, precision="tf32x3")
    from paper_2011_04240_b300 import amto
    assert pl.info.multipliers == amto.MULT_AGGREGATE
    yield pl, probs
    pl.close()


def test_sampled_instances_match_the_oracle(bench_plan):
    pl, probs = bench_plan
    k = 2  # inside the shell's parity horizon
    x, r, kk = gpu_solve(pl, probs, k)
    assert np.all(kk == k)
    M = oracle_mats(probs[0])
    for i in SAMPLES:
        st = oracle_solve(M, probs[i], k, mode="R3")
        assert rel_inf(x[i].reshape(3, -1), st.xi) < XI_TOL, i


def test_properties_at_the_benchmark_iteration_count(bench_plan):
    pl, probs = bench_plan
    K = 20
    x, r, kk = gpu_solve(pl, probs, K)
    assert np.all(kk == K)
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(r))
    M = oracle_mats(probs[0])
    for i in SAMPLES:
        xi = x[i].reshape(3, -1).astype(np.float64)
        # boundary conditions: A_eq xi = b_eq on every axis
        beq = O.boundary_values(probs[i].start, probs[i].goal, M.bc_mask)
        for ax in range(3):
            lhs = M.A_eq @ xi[ax]
            scale = np.abs(M.A_eq) @ np.abs(xi[ax])
            assert np.all(np.abs(lhs - beq[ax]) <= 1e-4 * scale + 1e-4), (i, ax)
        # the reported residual: the FP64 maximum over pairs and samples of
        # ||f_c|| at the returned iterate (lambda-free reading)
        D = O.pair_differences(M, xi)
        _, _, dd, U = O.projection(D, np.zeros_like(D), M, "R3")
        ref = O.residual_max(D - dd * U)
        assert abs(r[i] - ref) <= 1e-5 * max(ref, 1e-3), (i, r[i], ref)
    # one instance alone, with the same plan: the same bits as inside the batch
    xs, rs, ks = gpu_solve(pl, [probs[85]], K)
    assert np.array_equal(xs[0].view(np.uint32), x[85].view(np.uint32))
    assert np.array_equal(rs.view(np.uint32), r[85:86].view(np.uint32))
