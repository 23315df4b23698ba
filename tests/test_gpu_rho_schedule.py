"""Increasing-rho schedule on the GPU (Sec. IV-A; reading R-rho-sched).

QP solve k >= 1 uses rho_j = rho * g^j, j = min(J - 1, (k - 1) / E), with one
cached KKT inverse per stage and the multipliers carried over.  The CUDA path
must follow the oracle's `solve_schedule` across the stage switches (the
target of solve k + 1 is formed with rho of stage(k + 1), the multiplier
update of solve k with rho of stage(k)), in every loop and apply form; a
constant schedule must reproduce the plain solve bit for bit; and the paper's
point, fewer iterations to the residual tolerance, must hold on the GPU too.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import gpu_solve, rel_inf, to_dev

pytestmark = pytest.mark.gpu
MODES = {"R2": 0, "R3": 1}
XI_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _planner(prob, J, g, E, B=1, mode="R2", apply_mode=0, loop=0, precision=0):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree,
                   proj_mode=MODES[mode], max_batch=B, apply_mode=apply_mode, loop_mode=loop,
                   precision=precision, rho_stages=J, rho_growth=g, rho_stage_iters=E)


def _stage_mats(prob, J, g):
    return [O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b,
                             prob.rho * g ** j) for j in range(J)]


SMALL = W.random_box(8, 31, box=(5.0, 5.0, 2.5), m=40, T=5.0)


@pytest.mark.parametrize("loop,apply_mode,mode", [
    (1, 1, "R2"), (1, 2, "R2"), (1, 3, "R2"), (2, 1, "R2"), (2, 3, "R2"),
    (1, 1, "R3"), (2, 1, "R3")])
def test_schedule_matches_oracle_across_switches(loop, apply_mode, mode):
    J, g, E = 3, 3.0, 4
    Ms = _stage_mats(SMALL, J, g)
    pl = _planner(SMALL, J, g, E, mode=mode, apply_mode=apply_mode, loop=loop)
    assert pl.info.loop_mode == loop and pl.info.apply_mode == apply_mode
    for k in (E, E + 1, 2 * E + 1, 3 * E + 3):  # last of stage 0, first of 1 and 2, in 2
        x, r, kk = gpu_solve(pl, [SMALL], k)
        st = O.solve_schedule(Ms, E, SMALL.start, SMALL.goal, k, mode=mode)
        assert kk[0] == k
        assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, (k, rel_inf(x[0].reshape(3, -1), st.xi))
        assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2), (k, r[0], st.r_max)


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (2, 1e-3)])
def test_schedule_on_the_tensor_core_apply(precision, tol):
    """TF32x3 / BF16x3 apply: the tensor maps of the stage's inverse are chosen
    on the device from the stage the pair kernel left in the control block."""
    J, g, E = 3, 3.0, 3
    probs = [W.random_box(16, 40 + i, box=(6.0, 6.0, 3.0), m=60, T=6.0) for i in range(6)]
    Ms = _stage_mats(probs[0], J, g)
    pl = _planner(probs[0], J, g, E, B=6, precision=precision, loop=1)
    k = 2 * E + 2
    x, r, kk = gpu_solve(pl, probs, k)
    for i in (0, 5):
        st = O.solve_schedule(Ms, E, probs[i].start, probs[i].goal, k)
        assert rel_inf(x[i].reshape(3, -1), st.xi) < tol


def test_schedule_batched_16_agent_boxes():
    """16 agents, 6x6x3 m box, the schedule rho 1 -> 100 over ten stages of ten
    solves; a batch of eight through the batched GEMM apply."""
    J, g, E = 10, 100 ** (1 / 9), 10
    probs = [W.box16(i) for i in range(8)]
    Ms = _stage_mats(probs[0], J, g)
    pl = _planner(probs[0], J, g, E, B=8, loop=1, apply_mode=1)
    k = 23
    x, r, kk = gpu_solve(pl, probs, k)
    for i in (0, 7):
        st = O.solve_schedule(Ms, E, probs[i].start, probs[i].goal, k)
        assert rel_inf(x[i].reshape(3, -1), st.xi) < 5e-4


@pytest.mark.parametrize("loop,apply_mode", [(1, 1), (1, 2), (2, 1), (1, 3)])
def test_constant_schedule_is_the_plain_solve(loop, apply_mode):
    probs = [W.random_box(12, 50 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0) for i in range(3)]
    B = 3 if loop == 1 else 1
    ps = _planner(probs[0], 4, 1.0, 3, B=B, loop=loop, apply_mode=apply_mode)
    pp = _planner(probs[0], 0, 1.0, 1, B=B, loop=loop, apply_mode=apply_mode)
    xs, rs, ks = gpu_solve(ps, probs[:B], 17)
    xp, rp, kp = gpu_solve(pp, probs[:B], 17)
    assert np.array_equal(xs, xp) and np.array_equal(rs, rp) and np.array_equal(ks, kp)


def test_schedule_reaches_the_tolerance_sooner():
    """Sec. IV-A on the GPU: 16 agents in the 6x6x3 m box reach r_max < 1e-2 in
    fewer iterations with rho growing 1 -> 100 than at constant rho = 1, and
    the iteration count agrees with the oracle's."""
    prob = W.box16(0)
    J, g, E = 10, 100 ** (1 / 9), 10
    ps = _planner(prob, J, g, E, loop=1)
    pp = _planner(prob, 0, 1.0, 1, loop=1)
    _, rs, ks = gpu_solve(ps, [prob], 300, 1e-2)
    _, rp, kp = gpu_solve(pp, [prob], 300, 1e-2)
    assert rs[0] < 1e-2 and rp[0] < 1e-2
    assert ks[0] < 0.75 * kp[0], (ks[0], kp[0])
    st = O.solve_schedule(_stage_mats(prob, J, g), E, prob.start, prob.goal, 300, 1e-2)
    assert abs(int(ks[0]) - st.k) <= max(3, 0.05 * st.k), (ks[0], st.k)


def test_schedule_in_mixed_batches():
    from paper_2011_04240_b300 import Mixed, amto
    J, g, E = 3, 3.0, 4
    pa = [W.random_box(8, 70 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0) for i in range(3)]
    pb = [W.random_box(16, 80 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0) for i in range(2)]
    A = _planner(pa[0], J, g, E, B=3, loop=1)
    B = _planner(pb[0], J, g, E, B=2, loop=1)
    k = 2 * E + 1
    xa, _, _ = gpu_solve(A, pa, k)
    xb, _, _ = gpu_solve(B, pb, k)
    for layout in (amto.MIXED_FUSED, amto.MIXED_BRANCHES):
        mx = Mixed([A, B], layout)
        sa, ga = (to_dev(v, A.device) for v in W.stack(pa))
        sb, gb = (to_dev(v, A.device) for v in W.stack(pb))
        outs = mx.solve([sa, sb], [ga, gb], k)
        import torch
        torch.cuda.synchronize()
        (xma, _, kma), (xmb, _, kmb) = [(o[0].cpu().numpy(), o[1], o[2].cpu().numpy())
                                        for o in outs]
        assert (kma == k).all() and (kmb == k).all()
        assert rel_inf(xma, xa) < 2e-5 and rel_inf(xmb, xb) < 2e-5
        mx.close()
    # plans on different schedules cannot share one loop count
    C = _planner(pb[0], J, 2.0, E, B=2, loop=1)
    with pytest.raises(amto.AmtoError):
        Mixed([A, C])


def test_static_solve_follows_the_schedule():
    import torch
    from paper_2011_04240_b300 import amto
    lib = amto.load()
    J, g, E = 3, 3.0, 4
    pl = _planner(SMALL, J, g, E, loop=1)
    s = torch.from_numpy(SMALL.start[None]).cuda()
    gg = torch.from_numpy(SMALL.goal[None]).cuda()
    xi = torch.full((1, 3, SMALL.n, 11), float("nan"), device="cuda")
    r = torch.full((1,), float("nan"), device="cuda")
    k = torch.full((1,), -7, device="cuda", dtype=torch.int32)
    st = lib.amto_solve_static(pl.plan, s.data_ptr(), gg.data_ptr(), 2 * E + 1,
                               ctypes.c_float(0.0), xi.data_ptr(), r.data_ptr(), k.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.amto_last_error().decode()
    torch.cuda.synchronize()
    ref = O.solve_schedule(_stage_mats(SMALL, J, g), E, SMALL.start, SMALL.goal, 2 * E + 1)
    assert int(k[0]) == 2 * E + 1
    assert rel_inf(xi.cpu().numpy()[0].reshape(3, -1), ref.xi) < XI_TOL
