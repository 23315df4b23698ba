"""Python binding of the amto C ABI (include/amto.h): argument marshalling only.

Every step of the solver runs in the CUDA kernels of libamto.so.  This module
loads the in-tree library with ctypes and raises ImportError if it has not
been built; there is no other implementation to fall back to.

The low-level functions mirror the C entry points one to one (same names
without the ``amto_`` prefix) and take raw device pointers.  ``Planner`` is a
convenience wrapper that passes torch tensors' device pointers and the
current torch stream.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamto.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ENUMERIC, EPENDING = range(8)
PROJ_LITERAL, PROJ_NOLAMBDA = 0, 1
PREC_FP32, PREC_TF32X3, PREC_BF16X3, PREC_TF32, PREC_BF16, PREC_TF32_ADAPT, PREC_BF16_ADAPT = range(7)
APPLY_AUTO, APPLY_BATCHED, APPLY_FUSED, APPLY_KRONECKER = range(4)
LOOP_AUTO, LOOP_GRAPH, LOOP_BLOCK = range(3)
MULT_AUTO, MULT_PAIRS, MULT_AGGREGATE = range(3)
MIXED_FUSED, MIXED_BRANCHES, MIXED_LOOPS = range(3)
ADMIT_SHARED, ADMIT_FIXED = range(2)
BC_POS0, BC_VEL0, BC_ACC0, BC_POST, BC_VELT, BC_ACCT, BC_ALL = 1, 2, 4, 8, 16, 32, 63

STATUS_NAMES = {0: "AMTO_OK", 1: "AMTO_EINVAL", 2: "AMTO_ENOMEM", 3: "AMTO_ECUDA",
                4: "AMTO_ENONFINITE", 5: "AMTO_ETIMEOUT", 6: "AMTO_ENUMERIC", 7: "AMTO_EPENDING"}


class AmtoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int), ("m_steps", ctypes.c_int),
                ("poly_degree", ctypes.c_int), ("T", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("rho", ctypes.c_double),
                ("bc_mask", ctypes.c_uint), ("proj_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("tile_group", ctypes.c_int), ("tile_time_blocks", ctypes.c_int),
                ("apply_mode", ctypes.c_int), ("loop_mode", ctypes.c_int),
                ("rho_stages", ctypes.c_int), ("rho_growth", ctypes.c_double),
                ("rho_stage_iters", ctypes.c_int), ("multipliers", ctypes.c_int),
                ("n_obstacles", ctypes.c_int), ("planar", ctypes.c_int),
                ("prec_window", ctypes.c_int), ("prec_drop", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int), ("m_steps", ctypes.c_int), ("nv", ctypes.c_int),
                ("nb", ctypes.c_int), ("kkt_dim", ctypes.c_int), ("group", ctypes.c_int),
                ("t_chunk", ctypes.c_int), ("n_chunks", ctypes.c_int),
                ("lambda_floats", ctypes.c_longlong), ("kkt_check", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("launches_per_iteration", ctypes.c_int),
                ("launches_fixed", ctypes.c_int), ("time_blocks", ctypes.c_int),
                ("apply_mode", ctypes.c_int), ("loop_mode", ctypes.c_int),
                ("multipliers", ctypes.c_int), ("n_obstacles", ctypes.c_int),
                ("planar", ctypes.c_int), ("tuned", ctypes.c_int)]


class ServerParams(ctypes.Structure):
    _fields_ = [("n_sizes", ctypes.c_int), ("sizes", ctypes.POINTER(ctypes.c_int)),
                ("m_steps", ctypes.c_int), ("poly_degree", ctypes.c_int),
                ("T", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("rho", ctypes.c_double), ("proj_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_slots", ctypes.c_int),
                ("chunk_iters", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_float), ("memory_budget", ctypes.c_size_t),
                ("rho_stages", ctypes.c_int), ("rho_growth", ctypes.c_double),
                ("rho_stage_iters", ctypes.c_int), ("admission", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int), ("start", ctypes.c_void_p),
                ("goal", ctypes.c_void_p)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("resid", ctypes.c_float),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("iterations", ctypes.c_longlong),
                ("chunks", ctypes.c_longlong), ("n_groups", ctypes.c_int),
                ("sizes", ctypes.c_int * 32), ("slots", ctypes.c_int * 32),
                ("fair_slots", ctypes.c_int * 32), ("max_capacity", ctypes.c_int * 32),
                ("resizes", ctypes.c_longlong), ("budget", ctypes.c_size_t),
                ("budget_used", ctypes.c_size_t)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("tile_group", ctypes.c_int), ("tile_time_blocks", ctypes.c_int),
                ("apply_mode", ctypes.c_int), ("loop_mode", ctypes.c_int),
                ("us_per_iteration", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("n_entries", ctypes.c_int), ("entries", TuneEntry * 48), ("best", ctypes.c_int)]


_P = ctypes.c_void_p
SIGNATURES = {
    "amto_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "amto_destroy": (None, [_P]),
    "amto_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int,
                                  ctypes.c_float, _P, _P, _P, _P]),
    "amto_solve_static": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_float, _P, _P, _P,
                                         _P]),
    "amto_get_state": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "amto_get_aggregate": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "amto_solve_from_aggregate": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P,
                                                 ctypes.c_int, ctypes.c_float, _P, _P, _P, _P]),
    "amto_set_obstacles": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "amto_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "amto_get_kkt_inverse": (ctypes.c_int, [_P, _P]),
    "amto_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int)]),
    "amto_set_trace": (ctypes.c_int, [_P, ctypes.c_int]),
    "amto_tune": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(TuneResult)]),
    "amto_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "amto_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "amto_tune_cache_clear": (None, []),
    "amto_tune_cache_size": (ctypes.c_int, []),
    "amto_mixed_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(_P)]),
    "amto_mixed_solve": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_P),
                                        ctypes.POINTER(_P), ctypes.c_int, ctypes.c_float,
                                        ctypes.POINTER(_P), ctypes.POINTER(_P),
                                        ctypes.POINTER(_P), _P]),
    "amto_mixed_set_trace": (ctypes.c_int, [_P, ctypes.c_int]),
    "amto_mixed_destroy": (None, [_P]),
    "amto_server_create": (ctypes.c_int, [ctypes.POINTER(ServerParams), ctypes.POINTER(_P)]),
    "amto_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "amto_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, _P,
                                        ctypes.POINTER(ResultInfo)]),
    "amto_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "amto_admission_step": (ctypes.c_int, [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 5 +
                            [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_ulonglong,
                             ctypes.POINTER(ctypes.c_int)]),
    "amto_server_destroy": (None, [_P]),
    "amto_last_error": (ctypes.c_char_p, []),
    "amto_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libamto.so (once).  Raises ImportError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libamto.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise AmtoError(status, load().amto_last_error().decode())


def _ptr(x):
    """Device pointer of a torch tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# ----------------------------------------------------------------------------
# One-to-one wrappers of the C entry points
# ----------------------------------------------------------------------------

def create(params: Params) -> int:
    plan = _P()
    _check(load().amto_create(ctypes.byref(params), ctypes.byref(plan)))
    return plan.value


def destroy(plan: int) -> None:
    if plan:
        load().amto_destroy(plan)


def solve(plan, batch, start, goal, bc_extra, xi_init, lambda_init, max_iters, tol,
          xi_out, resid_out, iters_out, stream) -> None:
    _check(load().amto_solve(plan, batch, start, goal, bc_extra, xi_init, lambda_init,
                             max_iters, tol, xi_out, resid_out, iters_out, stream))


def solve_from_aggregate(plan, batch, start, goal, bc_extra, xi_init, agg_init, max_iters, tol,
                         xi_out, resid_out, iters_out, stream) -> None:
    _check(load().amto_solve_from_aggregate(plan, batch, start, goal, bc_extra, xi_init,
                                            agg_init, max_iters, tol, xi_out, resid_out,
                                            iters_out, stream))


def get_aggregate(plan, batch, agg_out, stream) -> None:
    _check(load().amto_get_aggregate(plan, batch, agg_out, stream))


def solve_static(plan, start, goal, max_iters, tol, xi_out, resid_out, iters_out,
                 stream) -> None:
    """One-instance solve whose scratch lives in the library's static device
    array (no allocation; see include/amto.h)."""
    _check(load().amto_solve_static(plan, start, goal, max_iters, tol, xi_out, resid_out,
                                    iters_out, stream))


def get_state(plan, batch, lambda_out, alpha_out, beta_out, d_out, stream) -> None:
    _check(load().amto_get_state(plan, batch, lambda_out, alpha_out, beta_out, d_out, stream))


def get_info(plan) -> Info:
    info = Info()
    _check(load().amto_get_info(plan, ctypes.byref(info)))
    return info


def get_kkt_inverse(plan, out_ptr) -> None:
    _check(load().amto_get_kkt_inverse(plan, out_ptr))


def get_stats(plan):
    ms = (ctypes.c_double * 3)()
    cnt = (ctypes.c_int * 3)()
    _check(load().amto_get_stats(plan, ms, cnt))
    return list(ms), list(cnt)


def set_trace(plan, on) -> None:
    """0/False: graph loop; 1/True: traced loop; 2: traced, L2 flushed before
    every iteration."""
    _check(load().amto_set_trace(plan, int(on)))


def tune(params: Params, batch: int, iters: int = 20) -> dict:
    """Measure the pair-kernel tiles (and apply and loop modes) for `params`
    on a synthetic batch; returns {"best": (tile_group, tile_time_blocks,
    apply_mode, loop_mode), "entries": [(G, QW, apply_mode, loop_mode,
    us/iteration)]}."""
    r = TuneResult()
    _check(load().amto_tune(ctypes.byref(params), int(batch), int(iters), ctypes.byref(r)))
    ent = [(r.entries[i].tile_group, r.entries[i].tile_time_blocks, r.entries[i].apply_mode,
            r.entries[i].loop_mode, r.entries[i].us_per_iteration) for i in range(r.n_entries)]
    return {"best": ent[r.best][:4], "entries": ent}


def admission_step(slots, active, queued, fair_slots, max_capacity, bytes_per_instance,
                   budget: int) -> list:
    """One step of the server's shared-budget admission policy on a description
    of the served counts (no device work); returns the capacities after it."""
    k = len(slots)
    ints = lambda v: (ctypes.c_int * k)(*[int(x) for x in v])  # noqa: E731
    out = (ctypes.c_int * k)()
    per = (ctypes.c_ulonglong * k)(*[int(x) for x in bytes_per_instance])
    _check(load().amto_admission_step(k, ints(slots), ints(active), ints(queued),
                                      ints(fair_slots), ints(max_capacity), per, int(budget), out))
    return list(out)


def tune_cache_save(path: str) -> None:
    """Write the tuning cache (amto_tune's best entry per shape) to `path`."""
    _check(load().amto_tune_cache_save(os.fsencode(path)))


def tune_cache_load(path: str) -> None:
    """Merge a file written by tune_cache_save into the tuning cache."""
    _check(load().amto_tune_cache_load(os.fsencode(path)))


def tune_cache_clear() -> None:
    load().amto_tune_cache_clear()


def tune_cache_size() -> int:
    return int(load().amto_tune_cache_size())


def last_error() -> str:
    return load().amto_last_error().decode()


def version() -> str:
    return load().amto_version().decode()


# ----------------------------------------------------------------------------
# torch convenience wrapper (device memory and streams only)
# ----------------------------------------------------------------------------

class Planner:
    """A plan for one agent count; solves batches of start/goal sets on the GPU.

    All tensors are float32 CUDA tensors on the plan's device.  Solves run on
    torch's current stream unless `stream` is given.
    """

    def __init__(self, n_agents: int, m_steps: int, T: float, a: float = 0.6, b: float = 1.2,
                 rho: float = 1.0, poly_degree: int = 10, bc_mask: int = BC_ALL,
                 proj_mode: int = PROJ_LITERAL, precision: int = PREC_FP32,
                 max_batch: int = 1, tile_group: int = 0, tile_time_blocks: int = 0,
                 apply_mode: int = 0, loop_mode: int = 0, rho_stages: int = 0,
                 rho_growth: float = 1.0, rho_stage_iters: int = 1, multipliers: int = 0,
                 n_obstacles: int = 0, planar: int = 0, prec_window: int = 0,
                 prec_drop: float = 0.0):
        import torch
        self._torch = torch
        self.plan = None
        self.params = Params(n_agents, m_steps, poly_degree, T, a, b, rho, bc_mask,
                             proj_mode, precision, max_batch, tile_group, tile_time_blocks,
                             apply_mode, loop_mode, rho_stages, rho_growth, rho_stage_iters,
                             multipliers, n_obstacles, planar, prec_window, prec_drop)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.plan = create(self.params)
        self.info = get_info(self.plan)
        self.n, self.m, self.nv = n_agents, m_steps, poly_degree + 1
        self.p = n_agents * (n_agents - 1) // 2
        self.last_batch = 0

    def close(self):
        if self.plan:
            destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        s = stream if stream is not None else self._torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def _check_tensor(self, t, shape, name, dtype=None):
        torch = self._torch
        dtype = dtype or torch.float32
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"{name}: expected contiguous {dtype} CUDA tensor of shape {shape}, "
                             f"got {tuple(t.shape)} {t.dtype} on {t.device}")
        return t

    def solve(self, start, goal, max_iters: int, tol: float = 0.0, bc_extra=None,
              xi_init=None, lambda_init=None, out=None, stream=None):
        """Run Algorithm 1; returns (xi [B,3,n,nv], resid [B], iters [B])."""
        torch = self._torch
        B = start.shape[0]
        n, nv = self.n, self.nv
        self._check_tensor(start, (B, n, 3), "start")
        self._check_tensor(goal, (B, n, 3), "goal")
        self._check_tensor(bc_extra, (B, n, 2, 2, 3), "bc_extra")
        self._check_tensor(xi_init, (B, 3, n, nv), "xi_init")
        self._check_tensor(lambda_init, (B, 3, self.p, self.m), "lambda_init")
        if out is None:
            xi = torch.empty((B, 3, n, nv), device=self.device, dtype=torch.float32)
            resid = torch.empty((B,), device=self.device, dtype=torch.float32)
            iters = torch.empty((B,), device=self.device, dtype=torch.int32)
        else:
            xi, resid, iters = out
        solve(self.plan, B, _ptr(start), _ptr(goal), _ptr(bc_extra), _ptr(xi_init),
              _ptr(lambda_init), int(max_iters), float(tol), _ptr(xi), _ptr(resid),
              _ptr(iters), self._stream(stream))
        self.last_batch = B
        return xi, resid, iters

    def solve_from_aggregate(self, start, goal, agg_init, max_iters: int, tol: float = 0.0,
                             bc_extra=None, xi_init=None, out=None, stream=None):
        """amto_solve with warm-start multipliers A_fc^T lambda [B,3,n,nv]
        (aggregated plans); returns (xi, resid, iters)."""
        torch = self._torch
        B = start.shape[0]
        n, nv = self.n, self.nv
        self._check_tensor(start, (B, n, 3), "start")
        self._check_tensor(goal, (B, n, 3), "goal")
        self._check_tensor(bc_extra, (B, n, 2, 2, 3), "bc_extra")
        self._check_tensor(xi_init, (B, 3, n, nv), "xi_init")
        self._check_tensor(agg_init, (B, 3, n, nv), "agg_init")
        if out is None:
            xi = torch.empty((B, 3, n, nv), device=self.device, dtype=torch.float32)
            resid = torch.empty((B,), device=self.device, dtype=torch.float32)
            iters = torch.empty((B,), device=self.device, dtype=torch.int32)
        else:
            xi, resid, iters = out
        solve_from_aggregate(self.plan, B, _ptr(start), _ptr(goal), _ptr(bc_extra),
                             _ptr(xi_init), _ptr(agg_init), int(max_iters), float(tol), _ptr(xi),
                             _ptr(resid), _ptr(iters), self._stream(stream))
        self.last_batch = B
        return xi, resid, iters

    def aggregate(self, stream=None):
        """A_fc^T lambda [B,3,n,nv] of the last solve (aggregated plans)."""
        torch = self._torch
        out = torch.empty((self.last_batch, 3, self.n, self.nv), device=self.device,
                          dtype=torch.float32)
        get_aggregate(self.plan, self.last_batch, _ptr(out), self._stream(stream))
        return out

    def set_obstacles(self, obstacles, stream=None):
        """Static obstacles [B, n_obstacles, 5] (centre x, y, z, l_xy, l_z of the
        combined agent-obstacle spheroid) for the instances of later solves."""
        B = obstacles.shape[0]
        self._check_tensor(obstacles, (B, self.params.n_obstacles, 5), "obstacles")
        _check(load().amto_set_obstacles(self.plan, B, _ptr(obstacles), self._stream(stream)))

    def state(self, stream=None):
        """(lambda [B,3,p,m], alpha, beta, d [B,p,m]) of the last solve; lambda
        is None for a plan that keeps the multipliers aggregated."""
        torch = self._torch
        B = self.last_batch
        lam = None
        if self.info.multipliers != MULT_AGGREGATE:
            lam = torch.empty((B, 3, self.p, self.m), device=self.device, dtype=torch.float32)
        al = torch.empty((B, self.p, self.m), device=self.device, dtype=torch.float32)
        be = torch.empty_like(al)
        d = torch.empty_like(al)
        get_state(self.plan, B, _ptr(lam), _ptr(al), _ptr(be), _ptr(d), self._stream(stream))
        return lam, al, be, d

    def kkt_inverse(self):
        import numpy as np
        k = self.info.kkt_dim
        out = np.empty((k, k), dtype=np.float64)
        get_kkt_inverse(self.plan, out.ctypes.data)
        return out

    def set_trace(self, on):
        set_trace(self.plan, on)

    def stats(self):
        return get_stats(self.plan)


# ----------------------------------------------------------------------------
# Mixed batches (several agent counts iterated as one loop)
# ----------------------------------------------------------------------------

class Mixed:
    """Solve instances of several agent counts as one loop (amto_mixed_*).

    `planners` are Planner objects (distinct agent counts, same m, degree,
    T, a, b, rho, boundary mask and projection mode); they must outlive this
    object.  solve() takes one (start, goal) pair of CUDA tensors per planner
    ([B_g, n_g, 3] each) and returns one (xi, resid, iters) per planner.
    """

    def __init__(self, planners, layout: int = 0):
        import torch
        self._torch = torch
        self.planners = list(planners)
        arr = (_P * len(self.planners))(*[p.plan for p in self.planners])
        h = _P()
        _check(load().amto_mixed_create(arr, len(self.planners), int(layout), ctypes.byref(h)))
        self.handle = h.value

    def solve(self, starts, goals, max_iters: int, tol: float = 0.0, out=None, stream=None):
        torch = self._torch
        ng = len(self.planners)
        bs, outs = [], []
        for g, pl in enumerate(self.planners):
            B = starts[g].shape[0]
            pl._check_tensor(starts[g], (B, pl.n, 3), "start")
            pl._check_tensor(goals[g], (B, pl.n, 3), "goal")
            bs.append(B)
            if out is None:
                outs.append((torch.empty((B, 3, pl.n, pl.nv), device=pl.device),
                             torch.empty((B,), device=pl.device),
                             torch.empty((B,), device=pl.device, dtype=torch.int32)))
            else:
                outs.append(out[g])
        P = lambda xs: (_P * ng)(*[x.data_ptr() for x in xs])  # noqa: E731
        s = stream if stream is not None else torch.cuda.current_stream(self.planners[0].device)
        _check(load().amto_mixed_solve(self.handle, (ctypes.c_int * ng)(*bs), P(starts), P(goals),
                                       int(max_iters), float(tol), P([o[0] for o in outs]),
                                       P([o[1] for o in outs]), P([o[2] for o in outs]),
                                       s.cuda_stream))
        for pl, B in zip(self.planners, bs):
            pl.last_batch = B
        return outs

    def set_trace(self, on: bool):
        _check(load().amto_mixed_set_trace(self.handle, 1 if on else 0))

    def close(self):
        if getattr(self, "handle", None):
            load().amto_mixed_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Serving (continuous batching; host inputs and outputs)
# ----------------------------------------------------------------------------

class Server:
    """Continuous-batching server for requests of mixed agent counts.

    Inputs are host numpy arrays; the server copies them at submit time.
    poll() returns None while a request is running, else a dict with the
    trajectories (numpy [3, n, N+1]), iterations, FP64 residual and the
    submit / admission / completion times (seconds, monotonic clock).
    """

    def __init__(self, sizes, m_steps=100, T=8.0, a=0.6, b=1.2, rho=1.0, poly_degree=10,
                 proj_mode=PROJ_LITERAL, precision=PREC_FP32, max_slots=64, chunk_iters=8,
                 max_iters=2000, tol=1e-2, memory_budget=0, rho_stages=0, rho_growth=1.0,
                 rho_stage_iters=1, admission=0):
        import numpy as np
        self._np = np
        self.sizes = [int(x) for x in sizes]
        self.nv = poly_degree + 1
        arr = (ctypes.c_int * len(self.sizes))(*self.sizes)
        self._sizes_arr = arr
        prm = ServerParams(len(self.sizes), arr, m_steps, poly_degree, T, a, b, rho, proj_mode,
                           precision, max_slots, chunk_iters, max_iters, tol, memory_budget,
                           rho_stages, rho_growth, rho_stage_iters, admission)
        h = _P()
        _check(load().amto_server_create(ctypes.byref(prm), ctypes.byref(h)))
        self.handle = h.value
        self._n_of = {}

    def submit(self, start, goal) -> int:
        np = self._np
        s = np.ascontiguousarray(start, dtype=np.float32)
        g = np.ascontiguousarray(goal, dtype=np.float32)
        n = s.shape[0]
        req = Request(n, s.ctypes.data, g.ctypes.data)
        t = ctypes.c_uint64()
        _check(load().amto_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._n_of[t.value] = n
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        np = self._np
        n = self._n_of[ticket]
        xi = np.empty((3, n, self.nv), dtype=np.float32)
        info = ResultInfo()
        st = load().amto_server_poll(self.handle, ticket, int(wait_ms), xi.ctypes.data,
                                     ctypes.byref(info))
        if st == EPENDING:
            return None
        del self._n_of[ticket]
        if st not in (OK, ENONFINITE, ETIMEOUT):
            raise AmtoError(st, last_error())
        return {"status": st, "xi": xi, "iters": info.iters, "resid": info.resid,
                "t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done}

    def stats(self):
        s = ServerStats()
        _check(load().amto_server_stats(self.handle, ctypes.byref(s)))
        ng = s.n_groups
        return {"completed": s.completed, "iterations": s.iterations, "chunks": s.chunks,
                "slots": {s.sizes[i]: s.slots[i] for i in range(ng)},
                "fair_slots": {s.sizes[i]: s.fair_slots[i] for i in range(ng)},
                "max_capacity": {s.sizes[i]: s.max_capacity[i] for i in range(ng)},
                "resizes": s.resizes, "budget": s.budget, "budget_used": s.budget_used}

    def close(self):
        if getattr(self, "handle", None):
            load().amto_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
