"""The pair kernel's blocks take their (instance, chunk) units from a counter
in the plan's control block, which the setup kernel and each launch's last
block reset.  A unit's arithmetic does not depend on the block that runs it,
so repeated solves on one plan, at the full batch and at a prefix of it, after
a solve whose instances stopped at different iterations, must give the same
bits (the tensor-core apply's split over K is fixed by the plan's largest
batch, so a column's sums do not depend on the batch either).  The horizon
m = 50 leaves every instance a ragged last chunk, the units handed out last.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import gpu_solve, planner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _same(a, b):
    return all(np.array_equal(x, y, equal_nan=True) for x, y in zip(a, b))


@pytest.mark.parametrize("mult", ["aggregate", "pairs"])
def test_repeated_and_prefix_solves_are_bitwise_equal(mult):
    probs = [W.random_box(16, 900 + i, box=(6.0, 6.0, 3.0), m=50, T=5.0) for i in range(8)]
    pl = planner(probs[0], mode="R3", max_batch=8, precision="tf32x3", loop_mode=1,
                 multipliers=mult)
    first = gpu_solve(pl, probs, 12)
    assert (first[2] == 12).all()
    assert _same(gpu_solve(pl, probs, 12), first)
    prefix = gpu_solve(pl, probs[:3], 12)
    assert _same(prefix, tuple(v[:3] for v in first))
    # instances that stop at different iterations leave the counter as reset
    xt, rt, kt = gpu_solve(pl, probs, 300, 5e-2)
    assert (rt < 5e-2).all() and len(set(kt.tolist())) > 1
    assert _same(gpu_solve(pl, probs, 12), first)


def test_traced_loop_hands_out_the_same_units():
    """The host-driven traced loop launches the same kernels one by one."""
    probs = [W.random_box(16, 950 + i, box=(6.0, 6.0, 3.0), m=50, T=5.0) for i in range(5)]
    pl = planner(probs[0], mode="R3", max_batch=5, precision="tf32x3", loop_mode=1)
    graph = gpu_solve(pl, probs, 9)
    pl.set_trace(1)
    traced = gpu_solve(pl, probs, 9)
    pl.set_trace(0)
    assert _same(traced, graph)
