"""Open-loop load driver of the serving form (host side only).

``run_arrivals`` replays a list of timed requests against an ``amto.Server``
(continuous batching in libamto.so) and ``run_sequential`` replays the same
list against plain one-instance FP32 solves, one request at a time in arrival
order (the per-instance GPU path a caller without the server would use).  Both
return one record per request with its latency (completion minus arrival),
iterations and final FP64 residual, so the two can be compared at equal
residual.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import amto


def summarize(records, wall_s, cap=None):
    """p50/p99 latency (ms), throughput (instance-iterations/s, requests/s)
    and the residual spread of a list of request records."""
    lat = np.array([r["latency"] for r in records], dtype=np.float64) * 1e3
    its = np.array([r["iters"] for r in records], dtype=np.int64)
    res = np.array([r["resid"] for r in records], dtype=np.float64)
    return {
        "requests": len(records),
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "inst_iter_per_s": float(its[its > 0].sum() / wall_s) if wall_s > 0 else None,
        "req_per_s": len(records) / wall_s if wall_s > 0 else None,
        "mean_iters": float(its.mean()) if len(its) else None,
        "resid_max": float(res.max()) if len(res) else None,
        "resid_p50": float(np.median(res)) if len(res) else None,
        "frac_at_cap": float((its >= cap).mean()) if (cap and len(its)) else None,
    }


def run_arrivals(server: "amto.Server", arrivals, wait_ms: int = 1000, keep_xi: bool = True):
    """Submit each (t_s, start, goal) of ``arrivals`` (sorted by t_s) at its
    arrival time, relative to the call; collect every result.

    Latency is taken from the server's own clock (completion minus submit).
    Returns (records, wall_s), wall_s from the first arrival to the last
    completion."""
    tickets = []
    lock = threading.Lock()
    submitted = threading.Event()
    records = []

    def collect():
        i = 0
        while True:
            with lock:
                have = i < len(tickets)
                tk = tickets[i] if have else None
            if not have:
                if submitted.is_set():
                    with lock:
                        if i >= len(tickets):
                            return
                    continue
                time.sleep(0.0005)
                continue
            ticket, n = tk
            res = None
            while res is None:
                res = server.poll(ticket, wait_ms)
            res["n"] = n
            res["latency"] = res["t_done"] - res["t_submit"]
            if not keep_xi:
                del res["xi"]
            records.append(res)
            i += 1

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for t, start, goal in arrivals:
        d = t0 + t - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tk = server.submit(start, goal)
        with lock:
            tickets.append((tk, int(np.asarray(start).shape[0])))
    submitted.set()
    th.join()
    if not records:
        return records, 0.0
    first = min(r["t_submit"] for r in records)
    last = max(r["t_done"] for r in records)
    return records, last - first


def run_sequential(planners: dict, arrivals, max_iters: int, tol: float):
    """Plain per-instance path: requests are solved one at a time, in arrival
    order, each by one ``amto_solve`` of batch 1 on the plan of its agent
    count (FP32 apply), host inputs copied in and results copied out per
    request.  Latency counts the wait behind earlier requests."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    records = []
    t0 = time.perf_counter()
    for t, start, goal in arrivals:
        d = t0 + t - time.perf_counter()
        if d > 0:
            time.sleep(d)
        n = int(np.asarray(start).shape[0])
        pl = planners[n]
        s = torch.from_numpy(np.ascontiguousarray(start, np.float32)).reshape(1, n, 3).to(dev)
        g = torch.from_numpy(np.ascontiguousarray(goal, np.float32)).reshape(1, n, 3).to(dev)
        xi, r, k = pl.solve(s, g, max_iters, tol)
        xi_h, r_h, k_h = xi.cpu(), r.cpu(), k.cpu()   # synchronises
        t1 = time.perf_counter()
        records.append({"n": n, "xi": xi_h.numpy()[0], "iters": int(k_h[0]),
                        "resid": float(r_h[0]), "latency": t1 - (t0 + t),
                        "t_submit": t0 + t, "t_done": t1})
    wall = records[-1]["t_done"] - records[0]["t_submit"] if records else 0.0
    return records, wall
