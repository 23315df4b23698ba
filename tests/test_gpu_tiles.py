"""Pair-kernel tilings (lane group G, time blocks per warp QW) and the
autotuner.  A tiling only changes which lanes and blocks handle which pairs
and samples (and so the order of the segmented sums), never the method:
every tiling must match the FP64 oracle and the automatic tiling within the
float32 tolerance, multipliers included."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_solve, gpu_state, oracle_mats, oracle_solve, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _planner(prob, B, G=0, QW=0, mode=0, apply_mode=0, precision=0, loop_mode=1, multipliers=0):
    """Graph-loop plans (the tiles and apply modes under test are its)."""
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree, proj_mode=mode,
                   max_batch=B, tile_group=G, tile_time_blocks=QW, apply_mode=apply_mode,
                   precision=precision, loop_mode=loop_mode, multipliers=multipliers)


@pytest.mark.parametrize("n,m,G,QW", [(16, 100, 8, 1), (16, 100, 8, 4), (16, 100, 16, 2),
                                      (24, 100, 8, 2), (24, 100, 16, 1), (24, 37, 32, 3),
                                      (33, 100, 32, 2), (64, 100, 16, 1), (64, 60, 32, 4),
                                      (5, 41, 8, 8), (2, 50, 8, 5)])
def test_tiling_matches_oracle_and_automatic(n, m, G, QW):
    probs = [W.random_box(n, 4000 + 7 * n + i, box=(8.0, 8.0, 4.0), m=m, T=6.0) for i in range(3)]
    pt = _planner(probs[0], 3, G, QW)
    pa = _planner(probs[0], 3)
    assert pt.info.group == G and pt.info.time_blocks == QW
    xt, rt, kt = gpu_solve(pt, probs, 10)
    lt = gpu_state(pt)[0]
    xa, ra, ka = gpu_solve(pa, probs, 10)
    la = gpu_state(pa)[0]
    assert np.all(kt == 10)
    assert rel_inf(xt, xa) < 1e-5
    floor = max(np.abs(la).max(), 1e-2)
    assert np.abs(lt - la).max() / floor < 1e-4
    np.testing.assert_allclose(rt, ra, rtol=1e-4, atol=1e-6)
    st = oracle_solve(oracle_mats(probs[0]), probs[0], 10)
    assert rel_inf(xt[0].reshape(3, -1), st.xi) < 1e-4


def test_tune_measures_candidates():
    from paper_2011_04240_b300 import amto
    prob = W.random_box(16, 1, box=(8.0, 8.0, 4.0))
    p = amto.Params(16, 100, 10, 8.0, 0.6, 1.2, 1.0, 63, 0, 0, 8, 0, 0, 0, 0)
    try:
        res = amto.tune(p, 8, 5)
    finally:
        amto.tune_cache_clear()  # later tests create plans of this shape
    assert len(res["entries"]) >= 10
    assert {e[0] for e in res["entries"]} == {8, 16}
    assert {e[2] for e in res["entries"]} == {amto.APPLY_BATCHED, amto.APPLY_FUSED}
    assert {e[3] for e in res["entries"]} == {amto.LOOP_GRAPH, amto.LOOP_BLOCK}
    assert all(e[4] > 0 for e in res["entries"])
    assert res["best"] in [e[:4] for e in res["entries"]]
    G, QW, mode, loop = res["best"]
    pl = _planner(prob, 2, G, QW, apply_mode=mode)
    x, r, k = gpu_solve(pl, [prob, prob], 3)
    assert np.all(k == 3)


@pytest.mark.parametrize("n,B,literal", [(16, 3, 0), (24, 2, 1), (64, 1, 0), (5, 4, 0)])
def test_fused_apply_equals_matrix_vector_kernel(n, B, literal):
    """The fused apply (right-hand side and K^-1 product in the pair kernel's
    last unit per instance) does the arithmetic of the stand-alone kernels:
    with batches of at most 4 (matrix-vector kernel) results are bitwise
    equal, iteration counts and final residuals included."""
    from paper_2011_04240_b300 import amto
    probs = [W.random_box(n, 6100 + 5 * n + i, box=(8.0, 8.0, 4.0)) for i in range(B)]
    pf = _planner(probs[0], B, mode=literal, apply_mode=amto.APPLY_FUSED)
    # the fused apply keeps the multipliers per pair: compare with the same form
    pb = _planner(probs[0], B, mode=literal, apply_mode=amto.APPLY_BATCHED,
                  multipliers=amto.MULT_PAIRS)
    assert pf.info.apply_mode == amto.APPLY_FUSED and pf.info.launches_per_iteration == 1
    assert pb.info.apply_mode == amto.APPLY_BATCHED
    xf, rf, kf = gpu_solve(pf, probs, 300, tol=1e-2)
    xb, rb, kb = gpu_solve(pb, probs, 300, tol=1e-2)
    assert np.array_equal(kf, kb)
    assert np.array_equal(xf, xb)
    assert np.array_equal(rf, rb)


def test_fused_apply_tracks_batched_gemm():
    from paper_2011_04240_b300 import amto
    probs = [W.random_box(32, 6500 + i, box=(8.0, 8.0, 4.0)) for i in range(12)]
    pf = _planner(probs[0], 12, apply_mode=amto.APPLY_FUSED)
    pb = _planner(probs[0], 12, apply_mode=amto.APPLY_BATCHED)
    xf, rf, kf = gpu_solve(pf, probs, 20)
    xb, rb, kb = gpu_solve(pb, probs, 20)
    # different summation orders of the K^-1 product (lane-strided rows vs
    # split-K tiles), amplified over 20 iterations
    assert rel_inf(xf, xb) < 5e-5
    st = oracle_solve(oracle_mats(probs[0]), probs[0], 20)
    assert rel_inf(xf[0].reshape(3, -1), st.xi) < 1e-4


def test_fused_apply_rejected_for_tensor_core_precisions():
    from paper_2011_04240_b300 import amto, AmtoError
    with pytest.raises(AmtoError):
        _planner(W.random_box(8, 1, box=(8.0, 8.0, 4.0)), 2, apply_mode=amto.APPLY_FUSED,
                 precision=amto.PREC_TF32X3)


def test_tuned_choice_drives_automatic_plans(tmp_path):
    """amto_tune keeps its best entry; a later plan of the same shape with an
    automatic tile, apply and loop takes it (amto_info.tuned), a plan of
    another batch size or with an explicit tile does not, and the choice
    survives a save / clear / load round trip.  The tuned plan still matches
    the automatic one within the float32 tolerance."""
    from paper_2011_04240_b300 import amto
    amto.tune_cache_clear()
    probs = [W.random_box(24, 8100 + i, box=(8.0, 8.0, 4.0)) for i in range(8)]
    try:
        p = amto.Params(24, 100, 10, 8.0, 0.6, 1.2, 1.0, 63, 0, 0, 8, 0, 0, 0, 0)
        res = amto.tune(p, 8, 5)
        G, QW, mode, loop = res["best"]
        assert amto.tune_cache_size() == 1

        def check(pl):
            assert pl.info.tuned == 1 and pl.info.loop_mode == loop
            if loop == amto.LOOP_GRAPH:
                assert (pl.info.group, pl.info.time_blocks, pl.info.apply_mode) == (G, QW, mode)

        pt = _planner(probs[0], 8, loop_mode=0)
        check(pt)
        # batch 5 rounds up to the same bucket (8); 32 and an explicit tile do not match
        check(_planner(probs[0], 5, loop_mode=0))
        assert _planner(probs[0], 32, loop_mode=0).info.tuned == 0
        assert _planner(probs[0], 8, G=8, QW=1, loop_mode=0).info.tuned == 0
        f = tmp_path / "tune.txt"
        amto.tune_cache_save(str(f))
        amto.tune_cache_clear()
        pa = _planner(probs[0], 8, loop_mode=0)
        assert pa.info.tuned == 0
        amto.tune_cache_load(str(f))
        check(_planner(probs[0], 8, loop_mode=0))
        xt, rt, kt = gpu_solve(pt, probs, 10)
        xa, ra, ka = gpu_solve(pa, probs, 10)
        assert np.all(kt == 10) and rel_inf(xt, xa) < 1e-5
    finally:
        amto.tune_cache_clear()
