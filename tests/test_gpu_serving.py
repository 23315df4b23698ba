"""Serving form: continuous batching of mixed agent counts (amto_server_*).

Requests are admitted into resident slots between iteration chunks while
other requests keep iterating; each result must be the same alone and in a
mix (every instance's arithmetic depends only on its own inputs and the
shared plan), must match the FP64 oracle at a fixed iteration count, and
must stop by the rule of Algorithm 1 (residual below tol, or max_iters).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import oracle_mats, oracle_solve, planner, gpu_solve, rel_inf

pytestmark = pytest.mark.gpu
PREC = {"fp32": 0, "tf32x3": 1}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _server(sizes, precision="fp32", **kw):
    from paper_2011_04240_b300 import Server
    base = dict(m_steps=100, T=8.0, proj_mode=0, precision=PREC[precision], max_slots=8,
                chunk_iters=4, max_iters=300, tol=1e-2)
    base.update(kw)
    return Server(sizes, **base)


def _collect(sv, tickets):
    out = {}
    for t in tickets:
        r = None
        while r is None:
            r = sv.poll(t, 2000)
        out[t] = r
    return out


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("slots", [8, 20])
def test_same_result_alone_and_in_mix(precision, slots):
    """slots = 20: chunks launch over slot prefixes of 8, 16 or 20 as the
    occupancy changes; the probe's result must not depend on which."""
    sizes = (8, 16, 24)
    sv = _server(sizes, precision, max_slots=slots)
    try:
        probe = W.random_box(16, 4242, box=(8.0, 8.0, 4.0))
        alone = _collect(sv, [sv.submit(probe.start, probe.goal)])
        (ra,) = alone.values()
        mix = [W.random_box(int(sizes[i % 3]), 7000 + i, box=(8.0, 8.0, 4.0)) for i in range(30)]
        tickets = [sv.submit(p.start, p.goal) for p in mix[:17]]
        # the probe arrives while the first requests are resident and iterating
        tp = sv.submit(probe.start, probe.goal)
        tickets += [sv.submit(p.start, p.goal) for p in mix[17:]]
        res = _collect(sv, tickets + [tp])
        rm = res[tp]
        assert rm["iters"] == ra["iters"]
        assert rel_inf(rm["xi"], ra["xi"]) <= 1e-6
        assert abs(rm["resid"] - ra["resid"]) <= 1e-6 * max(1.0, abs(ra["resid"]))
        # every request finished by the stopping rule, and was admitted after submit
        for t in tickets:
            r = res[t]
            assert r["status"] == 0
            assert 1 <= r["iters"] <= 300
            assert r["iters"] == 300 or r["resid"] < 1e-2 * 1.5
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        st = sv.stats()
        assert st["completed"] == 32
        assert set(st["slots"]) == set(sizes)
    finally:
        sv.close()


def test_fixed_iterations_match_oracle_and_batch_solve():
    """tol = 0: every request runs exactly max_iters iterations; compare with
    the FP64 oracle (xi parity tolerance) and the batched plain solve."""
    sv = _server((5, 12), "fp32", max_iters=10, tol=0.0, chunk_iters=3)
    try:
        probs = [W.random_box(5 if i % 2 else 12, 900 + i, box=(8.0, 8.0, 4.0)) for i in range(8)]
        tk = [sv.submit(p.start, p.goal) for p in probs]
        res = _collect(sv, tk)
        for t, p in zip(tk, probs):
            r = res[t]
            assert r["iters"] == 10
            st = oracle_solve(oracle_mats(p), p, 10)
            assert rel_inf(r["xi"].reshape(3, -1), st.xi) < 1e-4
        p = probs[1]
        xs, _, ks = gpu_solve(planner(p, max_batch=1), [p], 10)
        assert ks[0] == 10
        assert rel_inf(res[tk[1]]["xi"], xs[0]) < 1e-5
    finally:
        sv.close()


def test_rho_schedule_per_request():
    """Increasing rho in the server: each request follows the schedule from its
    own QP count although the slots are not in step (staggered submissions);
    results match the oracle's scheduled solve, and to the tolerance the
    requests need fewer iterations than at constant rho."""
    import time
    J, g, E = 4, 3.0, 3
    sv = _server((5, 12), "fp32", max_iters=11, tol=0.0, chunk_iters=2, rho_stages=J,
                 rho_growth=g, rho_stage_iters=E)
    try:
        probs = [W.random_box(5 if i % 2 else 12, 950 + i, box=(8.0, 8.0, 4.0)) for i in range(6)]
        tk = []
        for p in probs:
            tk.append(sv.submit(p.start, p.goal))
            time.sleep(0.002)  # let earlier requests run a chunk first
        res = _collect(sv, tk)
        for t, p in zip(tk, probs):
            Ms = [O.build_matrices(p.n, p.m, p.degree, p.T, p.a, p.b, p.rho * g ** j)
                  for j in range(J)]
            st = O.solve_schedule(Ms, E, p.start, p.goal, 11)
            assert res[t]["iters"] == 11
            assert rel_inf(res[t]["xi"].reshape(3, -1), st.xi) < 1e-4
    finally:
        sv.close()
    probs = [W.box16(i) for i in range(4)]
    iters = {}
    for sched in (False, True):
        kw = dict(rho_stages=10, rho_growth=100 ** (1 / 9), rho_stage_iters=10) if sched else {}
        sv = _server((16,), "fp32", max_iters=500, tol=1e-2, **kw)
        try:
            tk = [sv.submit(p.start, p.goal) for p in probs]
            res = _collect(sv, tk)
            assert all(res[t]["resid"] < 1e-2 * 1.001 for t in tk)
            iters[sched] = sum(res[t]["iters"] for t in tk)
        finally:
            sv.close()
    assert iters[True] < 0.75 * iters[False], iters


def test_memory_budget_sets_slots_and_queues():
    """A budget of about two instances per count: requests wait for free
    slots and still all complete."""
    from paper_2011_04240_b300 import Server, AmtoError
    from paper_2011_04240_b300.amto import ENOMEM
    with pytest.raises(AmtoError) as e:
        Server((8,), max_iters=20, memory_budget=1024)
    assert e.value.status == ENOMEM
    # about 0.38 MB of resident state per 16-agent instance, 0.11 MB per
    # 8-agent one: an 0.8 MB share holds two 16-agent slots
    sv = _server((8, 16), max_iters=20, tol=0.0, max_slots=1000, memory_budget=1_600_000)
    try:
        st = sv.stats()
        assert 1 <= st["slots"][16] <= 4 and 1 <= st["slots"][8] <= 16, st
        probs = [W.random_box(8 if i % 2 else 16, 50 + i, box=(8.0, 8.0, 4.0)) for i in range(12)]
        res = _collect(sv, [sv.submit(p.start, p.goal) for p in probs])
        assert all(r["iters"] == 20 for r in res.values())
        assert sv.stats()["completed"] == 12
    finally:
        sv.close()


def test_rejects_unserved_size_and_unknown_ticket():
    from paper_2011_04240_b300 import AmtoError
    from paper_2011_04240_b300 import amto as A
    sv = _server((8,), max_iters=5)
    try:
        p = W.random_box(16, 1, box=(8.0, 8.0, 4.0))
        with pytest.raises(AmtoError):
            sv.submit(p.start, p.goal)
        st = A.load().amto_server_poll(sv.handle, 987654321, 0, None, None)
        assert st == A.EINVAL
    finally:
        sv.close()


def _per_instance_bytes(n, precision="fp32", proj=0):
    """Device bytes of one resident instance, as the server accounts them."""
    sv = _server((n,), precision, proj_mode=proj, max_slots=4, memory_budget=1 << 30)
    try:
        st = sv.stats()
        return st["budget_used"] // st["slots"][n]
    finally:
        sv.close()


@pytest.mark.parametrize("precision,proj", [("fp32", 0), ("tf32x3", 1)])
def test_shared_budget_moves_capacity_without_changing_results(precision, proj):
    """Shared admission: a flooded count grows by taking the idle count's
    free slots, then the other way round; every request's result is bitwise
    the one of a server whose budget never forces a resize (the shape choices
    of both are fixed by the same largest capacity, 32 slots)."""
    kw = dict(proj_mode=proj, max_slots=32, chunk_iters=4, max_iters=60, tol=1e-2)
    per16 = _per_instance_bytes(16, precision, proj)
    tight = _server((8, 16), precision, memory_budget=40 * per16, **kw)
    roomy = _server((8, 16), precision, memory_budget=1 << 30, **kw)
    try:
        s0 = tight.stats()
        assert s0["fair_slots"][16] == 20 and s0["max_capacity"][16] == 32, s0
        assert s0["slots"][16] == 20 and s0["max_capacity"][8] == 32, s0
        assert roomy.stats()["slots"] == {8: 32, 16: 32}
        res = {}
        for phase, n in enumerate((16, 8)):
            probs = [W.random_box(n, 3000 + 100 * phase + i, box=(8.0, 8.0, 4.0))
                     for i in range(70)]
            out = []
            for sv in (tight, roomy):
                out.append(_collect(sv, [sv.submit(p.start, p.goal) for p in probs]))
            res[n] = out
            st = tight.stats()
            assert st["budget_used"] <= st["budget"], st
            if n == 16:
                assert st["slots"][16] == 32 and st["slots"][8] < 32, st
            else:
                assert st["slots"][8] > 8 and st["slots"][16] < 32, st
        assert tight.stats()["resizes"] >= 3
        assert roomy.stats()["resizes"] == 0
        for n, (a, b) in res.items():
            for (ta, ra), (tb, rb) in zip(a.items(), b.items()):
                assert ra["status"] == rb["status"] == 0
                assert ra["iters"] == rb["iters"]
                assert ra["resid"] == rb["resid"]
                assert np.array_equal(ra["xi"], rb["xi"]), (n, ta)
    finally:
        tight.close()
        roomy.close()


def test_fixed_admission_keeps_equal_shares():
    """AMTO_ADMIT_FIXED: a flooded count keeps its equal share."""
    from paper_2011_04240_b300.amto import ADMIT_FIXED
    per16 = _per_instance_bytes(16)
    sv = _server((8, 16), max_slots=32, max_iters=20, tol=0.0, memory_budget=40 * per16,
                 admission=ADMIT_FIXED)
    try:
        s0 = sv.stats()
        assert s0["slots"][16] == s0["max_capacity"][16] == 20, s0
        probs = [W.random_box(16, 4100 + i, box=(8.0, 8.0, 4.0)) for i in range(50)]
        res = _collect(sv, [sv.submit(p.start, p.goal) for p in probs])
        assert all(r["iters"] == 20 for r in res.values())
        st = sv.stats()
        assert st["resizes"] == 0 and st["slots"] == s0["slots"], st
    finally:
        sv.close()


def test_resize_keeps_rho_schedule_results():
    """Shared admission with the per-request rho schedule (structured apply,
    each slot at its own stage): results across resizes are bitwise those of
    a server that never resizes."""
    kw = dict(max_slots=16, chunk_iters=3, max_iters=12, tol=0.0, rho_stages=4,
              rho_growth=3.0, rho_stage_iters=3)
    per12 = _per_instance_bytes(12)
    tight = _server((5, 12), memory_budget=24 * per12, **kw)
    roomy = _server((5, 12), memory_budget=1 << 30, **kw)
    try:
        assert tight.stats()["slots"][12] < 16 and roomy.stats()["slots"] == {5: 16, 12: 16}
        probs = [W.random_box(12, 5200 + i, box=(8.0, 8.0, 4.0)) for i in range(40)]
        out = [_collect(sv, [sv.submit(p.start, p.goal) for p in probs]) for sv in (tight, roomy)]
        st = tight.stats()
        assert st["resizes"] >= 1 and st["slots"][12] == 16, st
        for ra, rb in zip(out[0].values(), out[1].values()):
            assert ra["iters"] == rb["iters"] == 12
            assert ra["resid"] == rb["resid"]
            assert np.array_equal(ra["xi"], rb["xi"])
    finally:
        tight.close()
        roomy.close()
