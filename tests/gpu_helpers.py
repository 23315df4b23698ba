"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
(via the ctypes binding) and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
import workloads as W

MODES = {"R2": 0, "R3": 1}


def rel_inf(a, b) -> float:
    """Normwise relative error max|a-b| / max|b| (the xi parity measure)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


PRECISIONS = {"fp32": 0, "tf32x3": 1, "bf16x3": 2, "tf32": 3, "bf16": 4, "tf32_adapt": 5,
              "bf16_adapt": 6}


MULT = {"auto": 0, "pairs": 1, "aggregate": 2}


def planner(prob: W.Problem, mode="R2", max_batch=1, bc_mask=63, precision="fp32",
            tile_group=0, tile_time_blocks=0, loop_mode=0, multipliers="auto",
            prec_window=0, prec_drop=0.0):
    from paper_2011_04240_b300 import Planner
    return Planner(prob.n, prob.m, prob.T, prob.a, prob.b, prob.rho, prob.degree,
                   bc_mask=bc_mask, proj_mode=MODES[mode], max_batch=max_batch,
                   precision=PRECISIONS[precision], tile_group=tile_group,
                   tile_time_blocks=tile_time_blocks, loop_mode=loop_mode,
                   multipliers=MULT[multipliers], prec_window=prec_window,
                   prec_drop=prec_drop)


def to_dev(x, dev):
    import torch
    if x is None:
        return None
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)


def gpu_solve(pl, probs, iters, tol=0.0, xi_init=None, lambda_init=None, bc_extra=None):
    """Solve the same-n problems `probs` as one batch; numpy results."""
    import torch
    s, g = W.stack(probs)
    dev = pl.device
    xi, r, k = pl.solve(to_dev(s, dev), to_dev(g, dev), iters, tol,
                        bc_extra=to_dev(bc_extra, dev), xi_init=to_dev(xi_init, dev),
                        lambda_init=to_dev(lambda_init, dev))
    torch.cuda.synchronize()
    return xi.cpu().numpy(), r.cpu().numpy(), k.cpu().numpy()


def gpu_state(pl):
    import torch
    lam, al, be, d = pl.state()
    torch.cuda.synchronize()
    lam = None if lam is None else lam.cpu().numpy()  # None: aggregated multipliers
    return lam, al.cpu().numpy(), be.cpu().numpy(), d.cpu().numpy()


def oracle_mats(prob: W.Problem, bc_mask=63):
    return O.build_matrices(prob.n, prob.m, prob.degree, prob.T, prob.a, prob.b, prob.rho,
                            bc_mask)


def oracle_solve(M, prob, iters, tol=0.0, mode="R2", state=None, bc_extra=None, history=None):
    return O.solve(M, prob.start, prob.goal, iters, tol, mode, bc_extra=bc_extra,
                   state=state, history=history)
