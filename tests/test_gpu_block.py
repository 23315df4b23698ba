"""One-block-per-instance solver (AMTO_LOOP_BLOCK): the whole loop of
Algorithm 1 for an instance in one thread block.  Same method and pair
arithmetic as the graph loop, per-agent sums in another order: results must
match the FP64 oracle (xi, residual) and the graph loop within the float32
tolerance, with the multiplier layout shared (state read-back, final FP64
residual, warm starts)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import (gpu_solve, gpu_state, oracle_mats, oracle_solve, rel_inf, to_dev)

pytestmark = pytest.mark.gpu
MODES = {"R2": 0, "R3": 1}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _planner(prob, B=1, mode="R2", loop=2, G=0, bc_mask=63):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree, bc_mask=bc_mask,
                   proj_mode=MODES[mode], max_batch=B, loop_mode=loop, tile_group=G)


@pytest.mark.parametrize("prob,k,mode,G", [
    (W.circle4_swap(), 10, "R2", 0), (W.circle4_swap(), 10, "R3", 0),
    (W.random_box(16, 5, box=(6.0, 6.0, 3.0)), 60, "R2", 0),
    (W.random_box(16, 6, box=(6.0, 6.0, 3.0)), 30, "R2", 8),
    (W.random_box(32, 7, box=(8.0, 8.0, 4.0)), 20, "R2", 0),
    (W.random_box(5, 8, m=37, T=4.0), 40, "R3", 0),
    (W.random_box(24, 9, box=(8.0, 8.0, 4.0), m=61, T=6.0), 15, "R2", 16)])
def test_block_matches_oracle(prob, k, mode, G):
    from paper_2011_04240_b300 import amto
    pl = _planner(prob, 1, mode, G=G)
    assert pl.info.loop_mode == amto.LOOP_BLOCK
    x, r, kk = gpu_solve(pl, [prob], k)
    assert kk[0] == k
    st = oracle_solve(oracle_mats(prob), prob, k, mode=mode)
    assert rel_inf(x[0].reshape(3, -1), st.xi) < 1e-4
    assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2)


@pytest.mark.parametrize("n,B", [(16, 5), (8, 12), (32, 3)])
def test_block_batch_matches_graph_loop(n, B):
    probs = [W.random_box(n, 300 + i, box=(8.0, 8.0, 4.0)) for i in range(B)]
    pb = _planner(probs[0], B, loop=2)
    pg = _planner(probs[0], B, loop=1)
    xb, rb, kb = gpu_solve(pb, probs, 400, tol=1e-2)
    lb = gpu_state(pb)
    xg, rg, kg = gpu_solve(pg, probs, 400, tol=1e-2)
    lg = gpu_state(pg)
    assert np.all(np.abs(kb - kg) <= 2), (kb, kg)
    same = kb == kg
    assert rel_inf(xb[same], xg[same]) < 2e-4
    fl = max(np.abs(lg[0]).max(), 1e-2)
    assert np.abs(lb[0][same] - lg[0][same]).max() / fl < 2e-3
    done = kb < 400
    assert np.all(rb[done] < 1e-2 * 1.001)


def test_block_reported_residual_is_the_maximum():
    probs = [W.random_box(16, 40 + i, box=(8.0, 8.0, 4.0)) for i in range(3)]
    pl = _planner(probs[0], 3)
    gpu_solve(pl, probs, 24)
    lam_a = gpu_state(pl)[0].astype(np.float64)
    x, r, k = gpu_solve(pl, probs, 25)
    lam_b = gpu_state(pl)[0].astype(np.float64)
    for i in range(3):
        ref = np.sqrt(((lam_b[i] - lam_a[i]) ** 2).sum(axis=0)).max()
        assert abs(r[i] - ref) <= 1e-6 * max(np.abs(lam_b[i]).max(), 1.0) + 1e-6 * ref


def test_block_warm_start_and_boundary_extras():
    prob = W.random_box(12, 77, box=(6.0, 6.0, 3.0))
    M = oracle_mats(prob)
    st10 = oracle_solve(M, prob, 10)
    xi0 = st10.xi.astype(np.float32).reshape(1, 3, 12, -1)
    p = 12 * 11 // 2
    lam0 = st10.lam.astype(np.float32).reshape(1, 3, p, prob.m)
    pl = _planner(prob)
    x, r, k = gpu_solve(pl, [prob], 5, xi_init=xi0, lambda_init=lam0)
    ws = O.warm_state(M, st10.xi, st10.lam)
    beq = O.boundary_values(prob.start, prob.goal)
    for _ in range(5):
        ws = O.am_iteration(M, ws, beq, "R2")
    assert rel_inf(x[0].reshape(3, -1), ws.xi) < 1e-4
    rng = np.random.default_rng(3)
    extra = (0.2 * rng.standard_normal((1, 12, 2, 2, 3))).astype(np.float32)
    pl2 = _planner(prob)
    x2, r2, k2 = gpu_solve(pl2, [prob], 8, bc_extra=extra)
    st = oracle_solve(M, prob, 8, bc_extra=extra[0].astype(np.float64))
    assert rel_inf(x2[0].reshape(3, -1), st.xi) < 1e-4


def test_block_rejects_unsupported_combinations():
    from paper_2011_04240_b300 import Planner, AmtoError, amto
    prob = W.random_box(8, 1, box=(8.0, 8.0, 4.0))
    with pytest.raises(AmtoError):
        Planner(8, 100, 8.0, max_batch=2, loop_mode=amto.LOOP_BLOCK, precision=amto.PREC_TF32X3)
    with pytest.raises(AmtoError):
        Planner(8, 100, 8.0, max_batch=2, loop_mode=amto.LOOP_BLOCK, apply_mode=amto.APPLY_FUSED)
