"""Structured apply of the cached KKT inverse (AMTO_APPLY_KRONECKER): the
exact agent structure K^-1 = I (x) K_n^-1 + (1/n) 1 1^T (x) (K_0^-1 - K_n^-1)
(pinned in the oracle's tests against its dense inverse) applied per agent.
Same method as the dense apply: results match the FP64 oracle and the dense
float32 apply within the float32 tolerance, in the graph loop, the block
solver and mixed batches."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_solve, oracle_mats, oracle_solve, rel_inf, to_dev

pytestmark = pytest.mark.gpu
MODES = {"R2": 0, "R3": 1}
KRON, DENSE = 3, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _planner(prob, B=1, mode="R2", apply_mode=KRON, loop=1, precision=0):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree,
                   proj_mode=MODES[mode], max_batch=B, apply_mode=apply_mode, loop_mode=loop,
                   precision=precision)


@pytest.mark.parametrize("prob,k,mode,loop", [
    (W.circle4_swap(), 10, "R2", 1), (W.circle4_swap(), 10, "R2", 2),
    (W.random_box(16, 21, box=(6.0, 6.0, 3.0)), 50, "R2", 1),
    (W.random_box(16, 22, box=(6.0, 6.0, 3.0)), 50, "R2", 2),
    (W.random_box(33, 23, box=(8.0, 8.0, 4.0), m=41, T=6.0), 20, "R3", 1),
    (W.shell_batch(1)[0], 1, "R3", 1)])
def test_kron_matches_oracle(prob, k, mode, loop):
    from paper_2011_04240_b300 import amto
    pl = _planner(prob, 1, mode, loop=loop)
    assert pl.info.apply_mode == amto.APPLY_KRONECKER
    x, r, kk = gpu_solve(pl, [prob], k)
    assert kk[0] == k
    st = oracle_solve(oracle_mats(prob), prob, k, mode=mode)
    assert rel_inf(x[0].reshape(3, -1), st.xi) < 1e-4
    assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2)


@pytest.mark.parametrize("n,B,precision", [(24, 10, 0), (64, 6, 1), (8, 5, 0)])
def test_kron_tracks_dense_apply(n, B, precision):
    probs = [W.random_box(n, 600 + i, box=(8.0, 8.0, 4.0)) for i in range(B)]
    pk = _planner(probs[0], B, apply_mode=KRON, precision=precision)
    pd = _planner(probs[0], B, apply_mode=DENSE)
    xk, rk, kk = gpu_solve(pk, probs, 10)
    xd, rd, kd = gpu_solve(pd, probs, 10)
    assert rel_inf(xk, xd) < 2e-5, rel_inf(xk, xd)


def test_kron_in_mixed_batches():
    from paper_2011_04240_b300 import Mixed
    sizes, batches = (8, 16, 24), (4, 3, 5)
    groups = [[W.random_box(n, 800 + 10 * n + i, box=(8.0, 8.0, 4.0)) for i in range(B)]
              for n, B in zip(sizes, batches)]
    pls = [_planner(gr[0], 8) for gr in groups]
    for layout in (0, 1):
        mx = Mixed(pls, layout)
        starts = [to_dev(W.stack(gr)[0], "cuda") for gr in groups]
        goals = [to_dev(W.stack(gr)[1], "cuda") for gr in groups]
        outs = mx.solve(starts, goals, 12)
        for g, gr in enumerate(groups):
            xs, rs, ks = gpu_solve(pls[g], gr, 12)
            assert rel_inf(outs[g][0].cpu().numpy(), xs) < 1e-6
        mx.close()
