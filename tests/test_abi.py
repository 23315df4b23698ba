"""CPU checks of the C ABI: the library loads, exports every function that
include/amto.h declares, and rejects invalid arguments before touching the
GPU (host-side validation only; no compute call needs a device here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amto.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amto_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_04240_b300 import amto
    return amto.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["amto_create", "amto_solve", "amto_destroy", "amto_get_state",
                     "amto_get_info", "amto_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2011_04240_b300 import amto
    assert set(_declared_functions()) <= set(amto.SIGNATURES)


def _params(**kw):
    from paper_2011_04240_b300 import amto
    base = dict(n_agents=4, m_steps=50, poly_degree=10, T=5.0, a=0.6, b=1.2, rho=1.0,
                bc_mask=63, proj_mode=0, precision=0, max_batch=1)
    base.update(kw)
    return amto.Params(**base)


@pytest.mark.parametrize("bad", [dict(n_agents=1), dict(n_agents=300), dict(m_steps=5),
                                 dict(poly_degree=1), dict(T=0.0), dict(a=-1.0),
                                 dict(b=float("nan")), dict(rho=0.0), dict(bc_mask=0b001000),
                                 dict(bc_mask=64 | 63), dict(proj_mode=7), dict(max_batch=0),
                                 dict(precision=9), dict(tile_group=12), dict(tile_group=4),
                                 dict(tile_time_blocks=-1), dict(tile_time_blocks=9),
                                 dict(n_agents=256, tile_group=8, tile_time_blocks=8),
                                 dict(apply_mode=4), dict(apply_mode=-1),
                                 dict(apply_mode=2, precision=1), dict(loop_mode=3),
                                 dict(loop_mode=2, precision=1), dict(loop_mode=2, apply_mode=2),
                                 dict(n_obstacles=-1), dict(n_obstacles=65),
                                 dict(n_obstacles=2, loop_mode=2),
                                 dict(n_obstacles=2, apply_mode=2),
                                 dict(multipliers=3), dict(multipliers=2, proj_mode=0),
                                 dict(rho_stages=17), dict(rho_stages=3, rho_growth=0.0),
                                 dict(planar=2), dict(planar=1, a=0.0)])
def test_create_rejects_invalid_params(lib, bad):
    from paper_2011_04240_b300 import amto
    plan = ctypes.c_void_p()
    st = lib.amto_create(ctypes.byref(_params(**bad)), ctypes.byref(plan))
    assert st == amto.EINVAL
    assert plan.value is None
    assert "invalid argument" in lib.amto_last_error().decode()


def test_null_arguments_rejected(lib):
    from paper_2011_04240_b300 import amto
    assert lib.amto_create(None, None) == amto.EINVAL
    assert lib.amto_solve(None, 1, None, None, None, None, None, 1, 0.0, None, None, None,
                          None) == amto.EINVAL
    assert lib.amto_get_info(None, None) == amto.EINVAL
    assert lib.amto_set_trace(None, 1) == amto.EINVAL
    assert lib.amto_set_obstacles(None, 1, None, None) == amto.EINVAL
    lib.amto_destroy(None)  # no-op
    assert lib.amto_version().decode().startswith("amto")


def _server_params(**kw):
    from paper_2011_04240_b300 import amto
    sizes = kw.pop("sizes", (8, 16))
    arr = (ctypes.c_int * len(sizes))(*sizes)
    base = dict(n_sizes=len(sizes), sizes=arr, m_steps=100, poly_degree=10, T=8.0, a=0.6,
                b=1.2, rho=1.0, proj_mode=0, precision=0, max_slots=8, chunk_iters=4,
                max_iters=100, tol=1e-2, memory_budget=0)
    base.update(kw)
    return amto.ServerParams(**base), arr


@pytest.mark.parametrize("bad", [dict(sizes=()), dict(sizes=(8, 8)), dict(sizes=(1,)),
                                 dict(sizes=(8, 300)), dict(chunk_iters=0), dict(max_iters=0),
                                 dict(tol=float("nan")), dict(max_slots=0), dict(m_steps=5),
                                 dict(precision=9), dict(proj_mode=3), dict(n_sizes=40),
                                 dict(admission=2)])
def test_server_create_rejects_invalid_params(lib, bad):
    """Checked before any device call, so this runs without a GPU."""
    from paper_2011_04240_b300 import amto
    prm, _keep = _server_params(**bad)
    h = ctypes.c_void_p()
    st = lib.amto_server_create(ctypes.byref(prm), ctypes.byref(h))
    assert st == amto.EINVAL
    assert h.value is None
    assert "invalid argument" in lib.amto_last_error().decode()


def test_server_null_arguments_rejected(lib):
    from paper_2011_04240_b300 import amto
    t = ctypes.c_uint64()
    assert lib.amto_server_create(None, None) == amto.EINVAL
    assert lib.amto_server_submit(None, None, ctypes.byref(t)) == amto.EINVAL
    assert lib.amto_server_poll(None, 1, 0, None, None) == amto.EINVAL
    assert lib.amto_server_stats(None, None) == amto.EINVAL
    lib.amto_server_destroy(None)  # no-op


def test_mixed_null_arguments_rejected(lib):
    from paper_2011_04240_b300 import amto
    h = ctypes.c_void_p()
    assert lib.amto_mixed_create(None, 1, 0, ctypes.byref(h)) == amto.EINVAL
    plans = (ctypes.c_void_p * 1)(None)
    assert lib.amto_mixed_create(plans, 1, 0, ctypes.byref(h)) == amto.EINVAL
    assert lib.amto_mixed_create(plans, 0, 0, ctypes.byref(h)) == amto.EINVAL
    assert lib.amto_mixed_create(plans, 9, 0, ctypes.byref(h)) == amto.EINVAL
    assert lib.amto_mixed_create(plans, 1, 2, ctypes.byref(h)) == amto.EINVAL
    assert lib.amto_mixed_solve(None, None, None, None, 1, 0.0, None, None, None,
                                None) == amto.EINVAL
    assert lib.amto_mixed_set_trace(None, 1) == amto.EINVAL
    lib.amto_mixed_destroy(None)  # no-op


def test_library_has_no_unresolved_internal_symbols():
    """Every internal function the library calls is defined in it (a symbol
    left undefined would only fail when first called on the GPU)."""
    import subprocess
    from paper_2011_04240_b300 import amto
    out = subprocess.run(["nm", "-C", "-u", amto.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    bad = [ln for ln in out.splitlines() if "amto" in ln]
    assert not bad, bad


def test_tune_rejects_invalid_arguments(lib):
    from paper_2011_04240_b300 import amto
    r = amto.TuneResult()
    assert lib.amto_tune(None, 1, 1, ctypes.byref(r)) == amto.EINVAL
    p = _params(max_batch=4)
    assert lib.amto_tune(ctypes.byref(p), 5, 10, ctypes.byref(r)) == amto.EINVAL
    assert lib.amto_tune(ctypes.byref(p), 0, 10, ctypes.byref(r)) == amto.EINVAL
    assert lib.amto_tune(ctypes.byref(p), 2, 0, ctypes.byref(r)) == amto.EINVAL
    bad = _params(n_agents=1)
    assert lib.amto_tune(ctypes.byref(bad), 1, 1, ctypes.byref(r)) == amto.EINVAL
