"""Mixed batches: instances of different agent counts iterated as one loop
(one right-hand-side launch, one grouped apply and one fused pair-step
launch per iteration for all agent counts; amto_mixed_*).

Per instance the arithmetic is that of the plan's own solve, so results must
match per-plan amto_solve runs, and the FP64 oracle at a fixed iteration
count; the stopping rule of Algorithm 1 acts per instance.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_solve, oracle_mats, oracle_solve, planner, rel_inf, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _groups(sizes, batches, seed0, box=(8.0, 8.0, 4.0)):
    return [[W.random_box(n, seed0 + 100 * n + i, box=box) for i in range(B)]
            for n, B in zip(sizes, batches)]


def _mixed_solve(mx, groups, iters, tol=0.0):
    import torch
    starts, goals = [], []
    for probs in groups:
        s, g = W.stack(probs)
        starts.append(to_dev(s, "cuda"))
        goals.append(to_dev(g, "cuda"))
    outs = mx.solve(starts, goals, iters, tol)
    torch.cuda.synchronize()
    return [(x.cpu().numpy(), r.cpu().numpy(), k.cpu().numpy()) for x, r, k in outs]


def _plan(prob, B, precision="fp32", apply_mode=0):
    """Plans in the graph loop: the per-plan reference solves then run the
    same kernels as the mixed loop."""
    from paper_2011_04240_b300 import Planner
    from tests.gpu_helpers import PRECISIONS
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree, max_batch=B,
                   precision=PRECISIONS[precision], apply_mode=apply_mode, loop_mode=1)


@pytest.mark.parametrize("precision,apply_mode,layout", [("fp32", 2, 0), ("fp32", 1, 0),
                                                          ("tf32x3", 0, 0), ("fp32", 0, 1),
                                                          ("tf32x3", 0, 1), ("fp32", 2, 1),
                                                          ("fp32", 0, 2), ("tf32x3", 0, 2),
                                                          ("fp32", 2, 2)])
def test_mixed_matches_per_plan_solves_and_oracle(precision, apply_mode, layout):
    """apply_mode 2: every group applies K^-1 inside the pair kernel (one
    launch per iteration); 1 (and 0 = automatic): grouped right-hand-side and
    GEMM launches (per-group tensor-core GEMMs for tf32x3).  layout 0: one
    fused pair launch over all groups; 1: per-group chains as parallel
    branches of the graph; 2: per-group loops as parallel branches (each
    group runs its own solve's kernels: bitwise the per-plan solve)."""
    from paper_2011_04240_b300 import Mixed
    sizes, batches = (8, 16, 24, 32, 5), (6, 5, 7, 5, 6)
    groups = _groups(sizes, batches, 11)
    pls = [_plan(gr[0], 8, precision, apply_mode) for gr in groups]
    mx = Mixed(pls, layout)
    res = _mixed_solve(mx, groups, 10)
    for g, probs in enumerate(groups):
        x, r, k = res[g]
        assert np.all(k == 10)
        xs, rs, ks = gpu_solve(pls[g], probs, 10)
        assert rel_inf(x, xs) < 1e-6, (sizes[g], rel_inf(x, xs))
        if layout == 2:
            assert np.array_equal(x, xs) and np.array_equal(r, rs)
        st = oracle_solve(oracle_mats(probs[0]), probs[0], 10)
        assert rel_inf(x[0].reshape(3, -1), st.xi) < 1e-4
    mx.close()


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_mixed_tolerance_stop_per_instance_and_trace_mode(layout):
    from paper_2011_04240_b300 import Mixed
    sizes, batches = (8, 16, 24, 32), (16, 16, 16, 16)
    groups = _groups(sizes, batches, 23)
    pls = [planner(gr[0], max_batch=16, loop_mode=1) for gr in groups]
    mx = Mixed(pls, layout)
    res = _mixed_solve(mx, groups, 500, tol=1e-2)
    mx.set_trace(True)
    res_t = _mixed_solve(mx, groups, 500, tol=1e-2)
    for g, probs in enumerate(groups):
        x, r, k = res[g]
        xt, rt, kt = res_t[g]
        assert np.array_equal(x, xt) and np.array_equal(k, kt)
        xs, rs, ks = gpu_solve(pls[g], probs, 500, tol=1e-2)
        assert np.all(np.abs(k - ks) <= 2), (sizes[g], k, ks)
        if layout == 2:  # each group's own loop: its own solve, stop included
            assert np.array_equal(k, ks) and np.array_equal(x, xs)
        done = k < 500
        assert np.all(r[done] < 1e-2 * 1.001)  # FP64 recheck of a float32 stop
        assert np.all(r[~done] >= 1e-2 * 0.999)
    mx.close()


def test_mixed_rejects_inconsistent_plans():
    from paper_2011_04240_b300 import Mixed, AmtoError
    a = planner(W.random_box(8, 1, box=(8.0, 8.0, 4.0)), max_batch=2)
    p = W.random_box(16, 2, box=(8.0, 8.0, 4.0), m=60)
    b = planner(p, max_batch=2)
    with pytest.raises(AmtoError):
        Mixed([a, b])
    with pytest.raises(AmtoError):
        Mixed([a, a])
