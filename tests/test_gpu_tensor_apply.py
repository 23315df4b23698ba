"""Parity of the tensor-core (tcgen05, TF32) cached-inverse apply.

The apply xi += K^-1_top [g ; e] (Eq. kkt_step_x) runs as one batched GEMM
on the tensor cores with float32 accumulation.  With the hi/lo split
(AMTO_PREC_TF32X3: hi*hi + hi*lo + lo*hi) it must track the float32 SIMT
path and the FP64 oracle within the float32 tolerance; plain TF32 (one
product) converges to other nearby solutions, so it is accepted on residual only.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import gpu_solve, oracle_mats, oracle_solve, planner, rel_inf

pytestmark = pytest.mark.gpu
XI_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_tf32x3_shell64_matches_oracle_and_fp32():
    probs = W.shell_batch(8)
    M = oracle_mats(probs[0])
    pt = planner(probs[0], "R3", max_batch=8, precision="tf32x3")
    pf = planner(probs[0], "R3", max_batch=8, precision="fp32")
    xt, rt, kt = gpu_solve(pt, probs, 1)
    for i, p in enumerate(probs[:3]):
        st = oracle_solve(M, p, 1, mode="R3")
        assert rel_inf(xt[i].reshape(3, -1), st.xi) < XI_TOL
    # the antipodal shell is chaotic (its parity horizon is 1-5 iterations), so
    # the split tensor-core and float32 SIMT applies are compared at k = 1 only;
    # multi-iteration tracking is checked on random boxes below
    xf, rf, kf = gpu_solve(pf, probs, 1)
    assert rel_inf(xt, xf) < 2e-5
    assert np.all(kt == 1)


@pytest.mark.parametrize("n,m,B", [(5, 30, 3), (16, 100, 64), (24, 40, 50)])
def test_tf32x3_partial_tiles_split_k_and_padding(n, m, B):
    """n = 5: kdim = 85 padded to 88, one 55-row tile; n = 16, B = 64: two
    row tiles, two column tiles, split over K; n = 24: uneven column tile."""
    probs = [W.random_box(n, 300 + i, box=(8.0, 8.0, 4.0), m=m, T=6.0) for i in range(B)]
    pt = planner(probs[0], max_batch=B, precision="tf32x3")
    pf = planner(probs[0], max_batch=B, precision="fp32")
    xt, rt, kt = gpu_solve(pt, probs, 10)
    xf, rf, kf = gpu_solve(pf, probs, 10)
    assert rel_inf(xt, xf) < 5e-5, rel_inf(xt, xf)
    M = oracle_mats(probs[0])
    for i in [0, B - 1]:
        st = oracle_solve(M, probs[i], 10)
        assert rel_inf(xt[i].reshape(3, -1), st.xi) < XI_TOL


def test_plain_tf32_runs_and_keeps_residual_scale():
    probs = W.shell_batch(4)
    pt = planner(probs[0], "R3", max_batch=4, precision="tf32")
    pf = planner(probs[0], "R3", max_batch=4, precision="fp32")
    xt, rt, kt = gpu_solve(pt, probs, 20)
    xf, rf, kf = gpu_solve(pf, probs, 20)
    assert np.all(np.isfinite(xt)) and np.all(kt == 20)
    assert np.all(rt < 2.0 * rf + 1e-3)


def test_bf16x3_one_apply_vs_oracle():
    """BF16 hi/lo split (about 16 significant bits per operand, the lo*lo
    product dropped): one iteration on the 64-agent shell stays within 1e-3
    of the FP64 oracle (measured about 1e-5, since the apply adds an
    increment to xi)."""
    probs = W.shell_batch(4)
    M = oracle_mats(probs[0])
    pb = planner(probs[0], "R3", max_batch=4, precision="bf16x3")
    xb, rb, kb = gpu_solve(pb, probs, 1)
    for i, p in enumerate(probs[:2]):
        st = oracle_solve(M, p, 1, mode="R3")
        assert rel_inf(xb[i].reshape(3, -1), st.xi) < 1e-3
    assert np.all(kb == 1)


@pytest.mark.parametrize("n,m,B", [(5, 30, 3), (24, 40, 50)])
def test_bf16x3_partial_tiles_track_fp32(n, m, B):
    probs = [W.random_box(n, 500 + i, box=(8.0, 8.0, 4.0), m=m, T=6.0) for i in range(B)]
    pb = planner(probs[0], max_batch=B, precision="bf16x3")
    pf = planner(probs[0], max_batch=B, precision="fp32")
    xb, rb, kb = gpu_solve(pb, probs, 10)
    xf, rf, kf = gpu_solve(pf, probs, 10)
    assert rel_inf(xb, xf) < 1e-3, rel_inf(xb, xf)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3", "tf32", "bf16"])
def test_mixed_precision_reaches_the_fp32_residual(precision):
    """Acceptance of the mixed applies on the residual: every instance that
    reaches tol in float32 reaches it too, with at most 5% more iterations
    in total for the split (x3) modes; the single-product modes converge to
    other nearby solutions and are accepted on the residual alone."""
    probs = [W.random_box(16, 700 + i, box=(6.0, 6.0, 3.0)) for i in range(16)]
    pf = planner(probs[0], max_batch=16, precision="fp32")
    pm = planner(probs[0], max_batch=16, precision=precision)
    xf, rf, kf = gpu_solve(pf, probs, 500, tol=1e-2)
    xm, rm, km = gpu_solve(pm, probs, 500, tol=1e-2)
    ok_f = rf < 1e-2
    assert ok_f.sum() >= 12
    assert np.all(np.isfinite(rm))
    if precision.endswith("x3"):
        assert np.all(rm[ok_f] < 1e-2 * 1.001)  # FP64 recheck of a float32 stop
        assert km[ok_f].sum() <= 1.05 * kf[ok_f].sum() + 2
    else:
        assert (rm < 1e-2).sum() >= ok_f.sum() - 1


# ---- per-instance precision switch (AMTO_PREC_*_ADAPT) ----------------------

@pytest.mark.parametrize("adapt,plain", [("tf32_adapt", "tf32"), ("bf16_adapt", "bf16")])
def test_switch_that_never_fires_is_the_single_product(adapt, plain):
    """With a stall window longer than the solve the correction never turns
    on: the switch mode is then the single-product mode bit for bit."""
    probs = [W.random_box(16, 720 + i, box=(6.0, 6.0, 3.0)) for i in range(5)]
    pa = planner(probs[0], max_batch=5, precision=adapt, prec_window=100000)
    pp = planner(probs[0], max_batch=5, precision=plain)
    xa, ra, ka = gpu_solve(pa, probs, 40)
    xp, rp, kp = gpu_solve(pp, probs, 40)
    assert np.array_equal(xa, xp) and np.array_equal(ra, rp)


@pytest.mark.parametrize("adapt", ["tf32_adapt", "bf16_adapt"])
def test_switch_is_per_instance(adapt):
    """An instance's iterates do not depend on the other instances of its
    batch (their switches decide only whether a tile runs the correction
    products; a column adds them only for its own switched instance)."""
    probs = [W.random_box(16, 740 + i, box=(6.0, 6.0, 3.0)) for i in range(6)]
    pa = planner(probs[0], max_batch=6, precision=adapt, prec_window=3, prec_drop=0.05)
    xb, rb, kb = gpu_solve(pa, probs, 400, tol=1e-2)
    for i in (0, 3, 5):
        xi, ri, ki = gpu_solve(pa, [probs[i]], 400, tol=1e-2)
        assert ki[0] == kb[i]
        assert np.array_equal(xi[0], xb[i]) and ri[0] == rb[i]


def test_switch_turns_on_the_correction():
    """A window of one iteration and a drop no iteration can meet switch every
    instance on after its second QP solve: from there on the iterates follow
    the split (x3) arithmetic, so after 10 iterations they are much closer to
    the float32 ones than the single product's are."""
    probs = [W.random_box(16, 760 + i, box=(6.0, 6.0, 3.0)) for i in range(4)]
    pa = planner(probs[0], max_batch=4, precision="tf32_adapt", prec_window=1, prec_drop=0.99)
    pp = planner(probs[0], max_batch=4, precision="tf32")
    pf = planner(probs[0], max_batch=4, precision="fp32")
    xa, _, _ = gpu_solve(pa, probs, 10)
    xp, _, _ = gpu_solve(pp, probs, 10)
    xf, _, _ = gpu_solve(pf, probs, 10)
    assert not np.array_equal(xa, xp)
    assert rel_inf(xa, xf) < 0.5 * rel_inf(xp, xf), (rel_inf(xa, xf), rel_inf(xp, xf))


@pytest.mark.parametrize("adapt", ["tf32_adapt", "bf16_adapt"])
def test_switch_reaches_the_fp32_residual(adapt):
    """The residual acceptance of the switch mode on the random-box set:
    every instance that reaches tol in float32 reaches it too (the FP64
    recheck of a float32 stop), and the iterations in total stay within
    5 % of float32's (measured: 1.012x for TF32, 0.83x for BF16)."""
    probs = [W.random_box(16, 700 + i, box=(6.0, 6.0, 3.0)) for i in range(16)]
    pf = planner(probs[0], max_batch=16, precision="fp32")
    pa = planner(probs[0], max_batch=16, precision=adapt)
    xf, rf, kf = gpu_solve(pf, probs, 500, tol=1e-2)
    xa, ra, ka = gpu_solve(pa, probs, 500, tol=1e-2)
    ok_f = rf < 1e-2
    assert ok_f.sum() >= 12
    assert np.all(ra[ok_f] < 1e-2 * 1.001)
    assert ka[ok_f].sum() <= 1.05 * kf[ok_f].sum() + 2, (ka[ok_f].sum(), kf[ok_f].sum())
