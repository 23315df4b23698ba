"""Aggregated multipliers (AMTO_MULT_AGGREGATE) in the lambda-free reading.

In that reading lambda enters an iteration only through b_fc (Eq. b_f), and
b_fc only through A_fc^T b_fc in the QP's right-hand side (Eq. kkt_step_x),
so the plan keeps L = A_fc^T lambda and updates it with the same linear map
as Eq. lag_update.  The iterates are the per-pair form's in exact arithmetic:
they must match the FP64 oracle (which keeps lambda per pair) within the
float32 tolerance, across rho-stage switches, warm starts, every apply and
precision, mixed batches, the server and the static solve; and the reported
residual must still be the FP64 maximum over all pairs and samples.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import (gpu_solve, gpu_state, oracle_mats, oracle_solve, planner,
                               rel_inf, to_dev)

pytestmark = pytest.mark.gpu
XI_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _amto():
    from paper_2011_04240_b300 import amto
    return amto


def test_automatic_choice_and_rejections():
    amto = _amto()
    prob = W.random_box(16, 3, box=(6.0, 6.0, 3.0), m=40, T=5.0)
    assert planner(prob, "R3").info.multipliers == amto.MULT_AGGREGATE
    assert planner(prob, "R3").info.lambda_floats == 0
    assert planner(prob, "R2").info.multipliers == amto.MULT_PAIRS
    assert planner(prob, "R3", multipliers="pairs").info.multipliers == amto.MULT_PAIRS
    small = W.random_box(6, 3, box=(5.0, 5.0, 2.5), m=30, T=4.0)
    pb = planner(small, "R3")  # automatic block solver keeps the per-pair form
    assert pb.info.loop_mode == amto.LOOP_BLOCK and pb.info.multipliers == amto.MULT_PAIRS
    pa = planner(small, "R3", multipliers="aggregate")  # automatic loop yields to it
    assert pa.info.loop_mode == amto.LOOP_GRAPH and pa.info.multipliers == amto.MULT_AGGREGATE
    with pytest.raises(amto.AmtoError):
        planner(prob, "R2", multipliers="aggregate")
    with pytest.raises(amto.AmtoError):
        planner(prob, "R3", loop_mode=2, multipliers="aggregate")
    from paper_2011_04240_b300 import Planner
    with pytest.raises(amto.AmtoError):
        Planner(prob.n, prob.m, prob.T, proj_mode=1, apply_mode=amto.APPLY_FUSED,
                multipliers=amto.MULT_AGGREGATE)
    # the fused apply keeps the per-pair form automatically
    pf = Planner(prob.n, prob.m, prob.T, proj_mode=1, apply_mode=amto.APPLY_FUSED)
    assert pf.info.multipliers == amto.MULT_PAIRS


@pytest.mark.parametrize("prob,k,precision", [
    (W.shell_batch(1)[0], 1, "fp32"), (W.shell_batch(1)[0], 3, "fp32"),
    (W.random_box(33, 23, box=(8.0, 8.0, 4.0), m=41, T=6.0), 30, "fp32"),
    (W.random_box(16, 21, box=(6.0, 6.0, 3.0)), 60, "fp32"),
    (W.random_box(24, 5, box=(8.0, 8.0, 4.0), m=57, T=6.0), 25, "tf32x3"),
    (W.random_box(2, 8, box=(3.0, 3.0, 2.0), m=20, T=3.0), 15, "fp32"),
    # 100 agents: lane group 8, 13 agent blocks (the last padded), paired own blocks
    (W.random_box(100, 31, box=(16.0, 16.0, 8.0)), 5, "fp32")])
def test_matches_oracle(prob, k, precision):
    amto = _amto()
    pl = planner(prob, "R3", precision=precision, loop_mode=1)
    assert pl.info.multipliers == amto.MULT_AGGREGATE
    x, r, kk = gpu_solve(pl, [prob], k)
    assert kk[0] == k
    st = oracle_solve(oracle_mats(prob), prob, k, mode="R3")
    assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, rel_inf(x[0].reshape(3, -1), st.xi)
    assert abs(r[0] - st.r_max) <= 1e-4 * max(st.r_max, 1e-2)


@pytest.mark.parametrize("n,B,precision,apply_mode,k", [
    (64, 8, "fp32", 0, 20), (64, 6, "tf32x3", 0, 10), (32, 12, "fp32", 3, 40),
    (24, 5, "bf16x3", 0, 10), (16, 40, "fp32", 0, 50),
    # lane group 16, four agent blocks: paired own blocks on four of six tiles
    (64, 64, "tf32x3", 0, 10),
    # lane group 8, 13 blocks (odd, the last padded): paired tiles with masks
    (100, 4, "fp32", 0, 10)])
def test_tracks_the_per_pair_form(n, B, precision, apply_mode, k):
    """Same batch through both forms: the float32 iterates agree to rounding.
    (Random boxes: on the antipodal sphere shell float32 rounding of either
    form grows about threefold per iteration, so both drift from the oracle
    alike after a few iterations; that case is compared at k <= 3 above.)"""
    from paper_2011_04240_b300 import Planner
    amto = _amto()
    box = (12.0, 12.0, 6.0) if n == 64 else (16.0, 16.0, 8.0) if n > 64 else (8.0, 8.0, 4.0)
    probs = [W.random_box(n, 700 + i, box=box) for i in range(B)]
    p0 = probs[0]
    prec = {"fp32": 0, "tf32x3": 1, "bf16x3": 2}[precision]
    mk = lambda mult: Planner(p0.n, p0.m, p0.T, p0.a, p0.b, p0.rho, p0.degree, proj_mode=1,  # noqa: E731
                              max_batch=B, precision=prec, apply_mode=apply_mode, loop_mode=1,
                              multipliers=mult)
    pa, pp = mk(amto.MULT_AGGREGATE), mk(amto.MULT_PAIRS)
    if n == 64 and B == 64:
        assert pa.info.group == 16
    if n == 100:
        assert pa.info.group == 8
    xa, ra, ka = gpu_solve(pa, probs, k)
    xp, rp, kp = gpu_solve(pp, probs, k)
    assert np.all(ka == k) and np.all(kp == k)
    tol = 1e-3 if precision == "bf16x3" else 5e-5
    assert rel_inf(xa, xp) < tol, rel_inf(xa, xp)
    np.testing.assert_allclose(ra, rp, rtol=1e-3, atol=1e-6)


def test_same_iterations_to_tolerance():
    probs = [W.random_box(16, 800 + i, box=(6.0, 6.0, 3.0)) for i in range(6)]
    pa = planner(probs[0], "R3", max_batch=6)
    pp = planner(probs[0], "R3", max_batch=6, multipliers="pairs")
    xa, ra, ka = gpu_solve(pa, probs, 400, 1e-2)
    xp, rp, kp = gpu_solve(pp, probs, 400, 1e-2)
    assert np.all(np.abs(ka - kp) <= 1), (ka, kp)
    done = ka < 400
    assert np.all(ra[done] < 1e-2 * 1.001)
    for i in range(2):
        st = oracle_solve(oracle_mats(probs[i]), probs[i], 400, 1e-2, mode="R3")
        assert abs(int(ka[i]) - st.k) <= 2


def test_rho_schedule():
    from paper_2011_04240_b300 import Planner
    prob = W.random_box(16, 31, box=(6.0, 6.0, 3.0), m=50, T=6.0)
    J, g, E = 3, 3.0, 4
    pl = Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree, proj_mode=1,
                 loop_mode=1, rho_stages=J, rho_growth=g, rho_stage_iters=E)
    assert pl.info.multipliers == _amto().MULT_AGGREGATE
    Ms = [O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b,
                           prob.rho * g ** j) for j in range(J)]
    for k in (E, E + 1, 2 * E + 1, 3 * E + 2):
        x, r, kk = gpu_solve(pl, [prob], k)
        st = O.solve_schedule(Ms, E, prob.start, prob.goal, k, mode="R3")
        assert rel_inf(x[0].reshape(3, -1), st.xi) < XI_TOL, k


@pytest.mark.parametrize("n,m,G", [(16, 100, 0), (24, 40, 32), (33, 17, 0)])
def test_warm_start_multipliers(n, m, G):
    """lambda_init is reduced to A_fc^T lambda in the setup: one iteration from
    the oracle's state after 15 iterations matches the oracle's next one."""
    prob = W.random_box(n, 40 + n, box=(6.0, 6.0, 3.0), m=m, T=6.0)
    M = oracle_mats(prob)
    st15 = oracle_solve(M, prob, 15, mode="R3")
    xi0 = st15.xi.astype(np.float32)
    lam0 = st15.lam.astype(np.float32)
    p = n * (n - 1) // 2
    ws = O.warm_state(M, xi0.astype(np.float64), lam0.astype(np.float64), "R3")
    beq = O.boundary_values(prob.start, prob.goal)
    ref1 = O.am_iteration(M, ws, beq, "R3")
    ref3 = O.am_iteration(M, O.am_iteration(M, ref1, beq, "R3"), beq, "R3")
    pl = planner(prob, "R3", tile_group=G, loop_mode=1)
    assert pl.info.multipliers == _amto().MULT_AGGREGATE
    for k, ref in ((1, ref1), (3, ref3)):
        xi, r, kk = gpu_solve(pl, [prob], k, xi_init=xi0.reshape(1, 3, n, -1),
                              lambda_init=lam0.reshape(1, 3, p, m))
        assert kk[0] == k
        assert rel_inf(xi[0].reshape(3, -1), ref.xi) < XI_TOL


def test_state_without_multipliers():
    amto = _amto()
    probs = [W.random_box(16, 60 + i, box=(6.0, 6.0, 3.0)) for i in range(2)]
    pa = planner(probs[0], "R3", max_batch=2)
    pp = planner(probs[0], "R3", max_batch=2, multipliers="pairs")
    gpu_solve(pa, probs, 7)
    gpu_solve(pp, probs, 7)
    lam, al, be, d = gpu_state(pa)
    assert lam is None
    _, al_p, be_p, d_p = gpu_state(pp)
    np.testing.assert_allclose(d, d_p, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(be, be_p, atol=1e-3)
    import torch
    buf = torch.empty((2, 3, pa.p, pa.m), device="cuda")
    with pytest.raises(amto.AmtoError):
        amto.get_state(pa.plan, 2, buf.data_ptr(), None, None, None,
                       torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("n,B,k", [(64, 2, 3), (16, 3, 40)])
def test_reported_residual_is_the_fp64_maximum(n, B, k):
    """With no per-pair multipliers to read back, recompute f_c of the
    lambda-free reading (Delta min(0, 1 - 1/s)) in FP64 from the returned
    float32 coefficients: its maximum is the reported residual."""
    probs = W.shell_batch(B) if n == 64 else \
        [W.random_box(n, 910 + i, box=(8.0, 8.0, 4.0)) for i in range(B)]
    pl = planner(probs[0], "R3", max_batch=B)
    x, r, kk = gpu_solve(pl, probs, k)
    M = oracle_mats(probs[0])
    for i in range(B):
        xi = x[i].reshape(3, -1).astype(np.float64)
        D = O.pair_differences(M, xi)
        _, _, dd, U = O.projection(D, np.zeros_like(D), M, "R3")
        ref = O.residual_max(D - dd * U)
        assert abs(r[i] - ref) <= 1e-5 * max(ref, 1e-3), (i, r[i], ref)


def test_mixed_batch_of_both_forms():
    from paper_2011_04240_b300 import Mixed
    amto = _amto()
    pa = [W.random_box(16, 70 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0) for i in range(3)]
    pb = [W.random_box(24, 80 + i, box=(6.0, 6.0, 3.0), m=50, T=6.0) for i in range(2)]
    A = planner(pa[0], "R3", max_batch=3, loop_mode=1)
    B = planner(pb[0], "R3", max_batch=2, loop_mode=1, multipliers="pairs")
    assert A.info.multipliers == amto.MULT_AGGREGATE and B.info.multipliers == amto.MULT_PAIRS
    k = 12
    xa, _, _ = gpu_solve(A, pa, k)
    xb, _, _ = gpu_solve(B, pb, k)
    import torch
    for layout in (amto.MIXED_FUSED, amto.MIXED_BRANCHES):
        mx = Mixed([A, B], layout)
        sa, ga = (to_dev(v, A.device) for v in W.stack(pa))
        sb, gb = (to_dev(v, A.device) for v in W.stack(pb))
        outs = mx.solve([sa, sb], [ga, gb], k)
        torch.cuda.synchronize()
        assert rel_inf(outs[0][0].cpu().numpy(), xa) < 2e-5
        assert rel_inf(outs[1][0].cpu().numpy(), xb) < 2e-5
        mx.close()


def test_server_lambda_free_plans():
    """The serving layer's lambda-free plans aggregate the multipliers; a
    request's fixed-iteration result matches the oracle."""
    from paper_2011_04240_b300 import Server
    sv = Server([16, 24], m_steps=40, T=5.0, proj_mode=1, max_slots=8, chunk_iters=4,
                max_iters=12, tol=0.0)
    probs = [W.random_box(16, 90, box=(6.0, 6.0, 3.0), m=40, T=5.0),
             W.random_box(24, 91, box=(6.0, 6.0, 3.0), m=40, T=5.0)]
    tks = [sv.submit(p.start, p.goal) for p in probs]
    for tk, p in zip(tks, probs):
        res = None
        while res is None:
            res = sv.poll(tk, 2000)
        assert res["iters"] == 12
        st = oracle_solve(oracle_mats(p), p, 12, mode="R3")
        assert rel_inf(np.asarray(res["xi"]).reshape(3, -1), st.xi) < XI_TOL
    sv.close()


def test_static_solve():
    import torch
    amto = _amto()
    lib = amto.load()
    prob = W.random_box(24, 5, box=(8.0, 8.0, 4.0))
    pl = planner(prob, "R3")
    assert pl.info.multipliers == amto.MULT_AGGREGATE
    s = torch.from_numpy(prob.start[None]).cuda()
    g = torch.from_numpy(prob.goal[None]).cuda()
    xi = torch.full((1, 3, prob.n, 11), float("nan"), device="cuda")
    r = torch.full((1,), float("nan"), device="cuda")
    k = torch.full((1,), -7, device="cuda", dtype=torch.int32)
    st = lib.amto_solve_static(pl.plan, s.data_ptr(), g.data_ptr(), 30, ctypes.c_float(0.0),
                               xi.data_ptr(), r.data_ptr(), k.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.amto_last_error().decode()
    torch.cuda.synchronize()
    xr, rr, kr = gpu_solve(pl, [prob], 30)
    assert int(k[0]) == 30
    assert rel_inf(xi.cpu().numpy(), xr) < XI_TOL


def _afc_t(M, lam):
    """A_fc^T lambda per axis, FP64: (3, n nv)."""
    p, m = M.n * (M.n - 1) // 2, M.m
    return np.stack([M.A_fc.T @ np.asarray(lam[a], np.float64).reshape(p * m) for a in range(3)])


def test_aggregate_read_back_matches_oracle_multipliers():
    """amto_get_aggregate returns A_fc^T lambda of Eq. (lag_update): after a
    warm start from the oracle's state at k = 15 (no iteration) it is that
    state's A_fc^T lambda, and after 1 and 3 more iterations the oracle's."""
    prob = W.random_box(16, 71, box=(6.0, 6.0, 3.0))
    M = oracle_mats(prob)
    st15 = oracle_solve(M, prob, 15, mode="R3")
    xi0, lam0 = st15.xi.astype(np.float32), st15.lam.astype(np.float32)
    ws = O.warm_state(M, xi0.astype(np.float64), lam0.astype(np.float64), "R3")
    beq = O.boundary_values(prob.start, prob.goal)
    refs = {0: ws}
    refs[1] = O.am_iteration(M, ws, beq, "R3")
    refs[3] = O.am_iteration(M, O.am_iteration(M, refs[1], beq, "R3"), beq, "R3")
    pl = planner(prob, "R3")
    assert pl.info.multipliers == _amto().MULT_AGGREGATE
    p = prob.n * (prob.n - 1) // 2
    for k, ref in refs.items():
        gpu_solve(pl, [prob], k, xi_init=xi0.reshape(1, 3, prob.n, -1),
                  lambda_init=lam0.reshape(1, 3, p, prob.m))
        agg = pl.aggregate().cpu().numpy()[0].reshape(3, -1)
        want = _afc_t(M, ref.lam)
        assert rel_inf(agg, want) < (1e-5 if k == 0 else 1e-4), (k, rel_inf(agg, want))


@pytest.mark.parametrize("planar", [0, 1])
def test_aggregate_round_trip_is_bitwise(planar):
    """Read (xi, A_fc^T lambda) after a solve and resume from them with no
    iteration: both come back bit for bit (the resume's initial projection
    updates no multiplier)."""
    import torch
    from paper_2011_04240_b300 import Planner
    probs = [W.random_box(24, 90 + i, box=(8.0, 8.0, 4.0)) for i in range(3)]
    p0 = probs[0]
    pl = Planner(p0.n, p0.m, p0.T, p0.a, p0.b, p0.rho, p0.degree, proj_mode=1, max_batch=3,
                 planar=planar)
    assert pl.info.multipliers == _amto().MULT_AGGREGATE
    s, g = W.stack(probs)
    s, g = torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda()
    xi1, r1, k1 = pl.solve(s, g, 9)
    agg1 = pl.aggregate()
    xi2, r2, k2 = pl.solve_from_aggregate(s, g, agg1.clone(), 0, xi_init=xi1.clone())
    agg2 = pl.aggregate()
    torch.cuda.synchronize()
    assert torch.equal(xi1, xi2) and torch.equal(agg1, agg2)
    assert np.all(k2.cpu().numpy() == 0)
    if planar:
        assert torch.all(agg1[:, 2] == 0)  # the plane has no z multipliers


def test_resume_from_aggregate_equals_lambda_init():
    """A warm start from A_fc^T lambda (formed here in FP64) follows the same
    iterates as one from the per-pair lambda it came from."""
    prob = W.random_box(16, 73, box=(6.0, 6.0, 3.0))
    M = oracle_mats(prob)
    st15 = oracle_solve(M, prob, 15, mode="R3")
    xi0, lam0 = st15.xi.astype(np.float32), st15.lam.astype(np.float32)
    import torch
    p = prob.n * (prob.n - 1) // 2
    pl = planner(prob, "R3")
    xa, ra, ka = gpu_solve(pl, [prob], 4, xi_init=xi0.reshape(1, 3, prob.n, -1),
                           lambda_init=lam0.reshape(1, 3, p, prob.m))
    agg = torch.from_numpy(np.ascontiguousarray(
        _afc_t(M, lam0).astype(np.float32).reshape(1, 3, prob.n, -1))).cuda()
    x0 = torch.from_numpy(np.ascontiguousarray(xi0.reshape(1, 3, prob.n, -1))).cuda()
    s, g = W.stack([prob])
    xb, rb, kb = pl.solve_from_aggregate(torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda(),
                                         agg, 4, xi_init=x0)
    torch.cuda.synchronize()
    assert int(kb[0]) == int(ka[0]) == 4
    assert rel_inf(xb.cpu().numpy(), xa) < 1e-5
    ref = O.solve(M, prob.start, prob.goal, 4, mode="R3",
                  state=O.warm_state(M, xi0.astype(np.float64), lam0.astype(np.float64), "R3"))
    assert rel_inf(xb.cpu().numpy()[0].reshape(3, -1), ref.xi) < XI_TOL


def test_aggregate_calls_reject_per_pair_plans():
    import torch
    amto = _amto()
    prob = W.random_box(8, 75, box=(6.0, 6.0, 3.0))
    pp = planner(prob, "R3", multipliers="pairs")
    gpu_solve(pp, [prob], 2)
    buf = torch.zeros((1, 3, 8, 11), device="cuda")
    with pytest.raises(amto.AmtoError):
        amto.get_aggregate(pp.plan, 1, buf.data_ptr(), None)
    s, g = W.stack([prob])
    with pytest.raises(amto.AmtoError):
        pp.solve_from_aggregate(torch.from_numpy(s).cuda(), torch.from_numpy(g).cuda(), buf, 1)
