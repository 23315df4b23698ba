"""GPU test of amto_solve_static, the one-instance solve that allocates nothing.

That entry point exists for callers that cannot call cudaMalloc while they
plan (a control loop with a fixed memory budget, a process whose device heap
belongs to its own pool allocator): it takes all per-solve scratch from one
static device array inside the library.  Its results must match amto_solve's
on the same plan and inputs within the float32 parity tolerance (it always
runs the graph loop's kernels with the one-instance matrix-vector apply, so
a plan whose amto_solve uses the batched split-K product or the one-block
loop sums in another order), and two calls in a row must both be right,
since every call reuses (and must re-clear) the same array.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import planner, rel_inf

pytestmark = pytest.mark.gpu
XI_TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2011_04240_b300 import amto
    return amto.load()


def _static_solve(lib, pl, prob, iters, tol):
    import torch
    s = torch.from_numpy(prob.start[None]).cuda()
    g = torch.from_numpy(prob.goal[None]).cuda()
    xi = torch.full((1, 3, prob.n, 11), float("nan"), device="cuda")
    r = torch.full((1,), float("nan"), device="cuda")
    k = torch.full((1,), -7, device="cuda", dtype=torch.int32)
    st = lib.amto_solve_static(pl.plan, s.data_ptr(), g.data_ptr(), iters, ctypes.c_float(tol),
                               xi.data_ptr(), r.data_ptr(), k.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.amto_last_error().decode()
    torch.cuda.synchronize()
    return xi.cpu().numpy(), r.cpu().numpy(), k.cpu().numpy()


def _regular_solve(pl, prob, iters, tol):
    import torch
    s = torch.from_numpy(prob.start[None]).cuda()
    g = torch.from_numpy(prob.goal[None]).cuda()
    xi, r, k = pl.solve(s, g, iters, tol)
    torch.cuda.synchronize()
    return xi.cpu().numpy(), r.cpu().numpy(), k.cpu().numpy()


def test_static_solve_matches_solve_on_two_calls_in_a_row(lib):
    probs = [W.box16(0), W.box16(1)]
    pl = planner(probs[0])
    for prob in probs:  # the second call reuses the array the first one left behind
        xs, rs, ks = _static_solve(lib, pl, prob, 500, 1e-2)
        xr, rr, kr = _regular_solve(pl, prob, 500, 1e-2)
        assert ks[0] == kr[0]
        assert rel_inf(xs, xr) < XI_TOL
        assert abs(rs[0] - rr[0]) <= 1e-4 * max(rr[0], 1e-6)
    # a fixed iteration count, and a different agent count on a second plan
    prob = W.random_box(24, 5, box=(8.0, 8.0, 4.0))
    pl2 = planner(prob, "R3")
    for _ in range(2):
        xs, rs, ks = _static_solve(lib, pl2, prob, 40, 0.0)
        xr, rr, kr = _regular_solve(pl2, prob, 40, 0.0)
        assert ks[0] == kr[0] == 40
        assert rel_inf(xs, xr) < XI_TOL


def test_static_solve_on_a_one_block_plan(lib):
    """A 4-agent float32 plan runs amto_solve in the one-block loop; the
    static solve runs the graph loop's kernels on it.  Within the circle's
    parity horizon (k <= 10) both follow the FP64 oracle."""
    import oracle as O
    from tests.gpu_helpers import oracle_mats, oracle_solve
    prob = W.circle4_swap()
    pl = planner(prob)
    assert pl.info.loop_mode == 2  # AMTO_LOOP_BLOCK
    M = oracle_mats(prob)
    for k in (3, 8):
        xs, rs, ks = _static_solve(lib, pl, prob, k, 0.0)
        xr, rr, kr = _regular_solve(pl, prob, k, 0.0)
        st = oracle_solve(M, prob, k)
        assert ks[0] == kr[0] == k
        assert rel_inf(xs[0].reshape(3, -1), st.xi) < XI_TOL
        assert rel_inf(xs, xr) < XI_TOL
        assert abs(rs[0] - st.r_max) <= 1e-3 * max(st.r_max, 1e-3)


def test_static_solve_on_a_batched_plan(lib):
    """A plan made for batches of 8 applies K^-1 in amto_solve by the split-K
    matrix product; the static solve's matrix-vector apply sums in another
    order, so the trajectories agree to the float32 tolerance (iteration
    counts are not compared)."""
    probs = [W.random_box(16, 40 + i, box=(8.0, 8.0, 4.0)) for i in range(2)]
    pl = planner(probs[0], max_batch=8)
    for prob in probs:
        xs, rs, ks = _static_solve(lib, pl, prob, 60, 0.0)
        xr, rr, kr = _regular_solve(pl, prob, 60, 0.0)
        assert ks[0] == kr[0] == 60
        assert rel_inf(xs, xr) < XI_TOL
        assert abs(rs[0] - rr[0]) <= 1e-3 * max(rr[0], 1e-3)


def test_static_solve_rejects_plans_beyond_its_array(lib):
    prob = W.Problem(n=96, m=100, T=8.0, start=np.zeros((96, 3), np.float32),
                     goal=np.zeros((96, 3), np.float32))
    pl = planner(prob)
    import torch
    buf = torch.zeros((1, 3, 96, 11), device="cuda")
    st = lib.amto_solve_static(pl.plan, buf.data_ptr(), buf.data_ptr(), 1, ctypes.c_float(0.0),
                               buf.data_ptr(), None, None, None)
    assert st == 1  # AMTO_EINVAL
    assert "bytes of scratch" in lib.amto_last_error().decode()
