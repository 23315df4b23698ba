"""Seeded synthetic start/goal generators for the multi-agent planning problems.

This module is shared by the FP64 oracle tests and the GPU path's tests and
benchmark.  It holds no arithmetic of the optimisation method itself: it only
draws positions.  Every generator works in float64 and rounds the result to
float32 once, so both sides of a parity test receive bit-identical inputs.

Benchmark families follow the paper's Section IV-B: agents swapping to
antipodal positions, and random start/goal positions sampled in a room.
The paper's own datasets are not used; these synthetic sets stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Problem constants shared by every workload (Section III, spheroid agents).
DEGREE = 10          # per-axis Bernstein degree: 11 coefficients per agent and axis
A_XY = 0.6           # spheroid semi-axis l_xy (m)
B_Z = 1.2            # spheroid semi-axis l_z (m)
RHO = 1.0            # augmented-Lagrangian weight
MIN_SEP = 1.2        # minimum start-start / goal-goal separation (m)


@dataclasses.dataclass
class Problem:
    """One planning instance: n agents, start/goal positions, horizon."""
    n: int
    m: int
    T: float
    start: np.ndarray      # (n, 3) float32
    goal: np.ndarray       # (n, 3) float32
    a: float = A_XY
    b: float = B_Z
    rho: float = RHO
    degree: int = DEGREE
    name: str = ""


def _f32(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))


def circle_swap(n: int = 4, radius: float = 3.0, z: float = 1.0,
                m: int = 50, T: float = 5.0) -> Problem:
    """Agents on a circle swap to antipodal points (square/circle benchmark).

    theta_i = 2*pi*i/n, start = (r cos, r sin, z), goal = (-x, -y, z) by exact
    negation of the float32 start, so the instance is exactly symmetric.
    """
    th = 2.0 * math.pi * np.arange(n) / n
    start = _f32(np.stack([radius * np.cos(th), radius * np.sin(th), np.full(n, z)], 1))
    goal = start.copy()
    goal[:, :2] = -start[:, :2]
    return Problem(n=n, m=m, T=T, start=start, goal=goal, name=f"circle{n}")


def offset_swap2(m: int = 50, T: float = 5.0) -> Problem:
    """Two agents swapping with a small lateral offset (a 2-agent swap)."""
    start = _f32([[-2.0, 0.1, 1.0], [2.0, -0.1, 1.0]])
    goal = _f32([[2.0, -0.1, 1.0], [-2.0, 0.1, 1.0]])
    return Problem(n=2, m=m, T=T, start=start, goal=goal, name="swap2")


def _reject_points(rng: np.random.Generator, n: int, lo, hi, min_sep: float,
                   max_tries: int = 200000) -> np.ndarray:
    """n points uniform in the box [lo, hi] with pairwise distance >= min_sep."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    pts = np.empty((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampler could not place all agents")
        c = lo + (hi - lo) * rng.random(3)
        if k == 0 or np.sqrt(((pts[:k] - c) ** 2).sum(axis=1)).min() >= min_sep:
            pts[k] = c
            k += 1
    return pts


def random_box(n: int, seed: int, box=(6.0, 6.0, 3.0), m: int = 100,
               T: float = 8.0, min_sep: float = MIN_SEP) -> Problem:
    """Starts and goals drawn independently, uniform in a box, rejection-sampled.

    numpy default_rng(seed); starts first, then goals; separation is enforced
    among the starts and among the goals.
    """
    rng = np.random.default_rng(seed)
    s = _reject_points(rng, n, (0, 0, 0), box, min_sep)
    g = _reject_points(rng, n, (0, 0, 0), box, min_sep)
    return Problem(n=n, m=m, T=T, start=_f32(s), goal=_f32(g),
                   name=f"box{n}_s{seed}")


def sphere_shell(n: int, seed: int, radius: float = 5.0, m: int = 100,
                 T: float = 8.0, min_sep: float = MIN_SEP) -> Problem:
    """Starts uniform on a sphere shell about the origin, goal = -start.

    Rejection keeps start-start and start-(other agent's goal) distances
    >= min_sep.
    """
    rng = np.random.default_rng(seed)
    pts = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("shell sampler could not place all agents")
        v = rng.standard_normal(3)
        v = radius * v / np.linalg.norm(v)
        ok = True
        for p in pts:
            if np.linalg.norm(v - p) < min_sep or np.linalg.norm(v + p) < min_sep:
                ok = False
                break
        if ok:
            pts.append(v)
    start = _f32(np.array(pts))
    goal = -start
    return Problem(n=n, m=m, T=T, start=start, goal=goal, name=f"shell{n}_s{seed}")


def obstacle_box(n: int, n_obs: int, seed: int, box=(6.0, 6.0, 3.0), m: int = 100,
                 T: float = 8.0, r_range=(0.3, 0.6), min_sep: float = MIN_SEP):
    """Random start/goal box with static spherical obstacles (the paper's
    random-obstacle benchmark, Sec. IV): obstacle centres uniform in the box,
    radii uniform in r_range; each obstacle row holds the centre and the
    semi-axes of the combined agent-obstacle spheroid (l_xy/2 + r, l_z/2 + r).
    Starts and goals are rejection-sampled like random_box and also kept 0.2 m
    outside every combined spheroid.  Returns (Problem, obstacles (n_obs, 5)
    float32)."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.asarray(box, np.float64)
    cen = lo + (hi - lo) * rng.random((n_obs, 3))
    rad = r_range[0] + (r_range[1] - r_range[0]) * rng.random(n_obs)
    ax = A_XY / 2 + rad
    bz = B_Z / 2 + rad

    def clear(c):
        if n_obs == 0:
            return True
        q = ((c[0] - cen[:, 0]) ** 2 + (c[1] - cen[:, 1]) ** 2) / (ax + 0.2) ** 2 + \
            (c[2] - cen[:, 2]) ** 2 / (bz + 0.2) ** 2
        return bool(q.min() >= 1.0)

    def sample():
        pts = np.empty((n, 3))
        k = tries = 0
        while k < n:
            tries += 1
            if tries > 200000:
                raise RuntimeError("obstacle sampler could not place all agents")
            c = lo + (hi - lo) * rng.random(3)
            if (k == 0 or np.sqrt(((pts[:k] - c) ** 2).sum(axis=1)).min() >= min_sep) and clear(c):
                pts[k] = c
                k += 1
        return pts

    s = sample()
    g = sample()
    ob = np.concatenate([cen, ax[:, None], bz[:, None]], axis=1)
    return (Problem(n=n, m=m, T=T, start=_f32(s), goal=_f32(g), name=f"obst{n}x{n_obs}_s{seed}"),
            _f32(ob))


# ---------------------------------------------------------------------------
# The five workload configurations.
# ---------------------------------------------------------------------------

def circle4_swap() -> Problem:
    """4 agents, circle of radius 3 m at z = 1 m, antipodal goals, m=50, T=5 s."""
    return circle_swap(4, 3.0, 1.0, m=50, T=5.0)


def box16(seed: int = 0) -> Problem:
    """16 agents in a 6x6x3 m box, m=100, T=8 s."""
    return random_box(16, seed, box=(6.0, 6.0, 3.0), m=100, T=8.0)


def mixed_boxes(n_instances: int = 512, seed: int = 0, sizes=(8, 16, 24, 32)) -> list[Problem]:
    """Mixed batch: agent counts uniform in `sizes`, 8x8x4 m box, m=100, T=8 s."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=n_instances)
    return [random_box(int(n), seed * 100003 + i, box=(8.0, 8.0, 4.0), m=100, T=8.0)
            for i, n in enumerate(ns)]


def shell_batch(n_instances: int = 256, seed: int = 0, n: int = 64) -> list[Problem]:
    """n agents each on a 5 m sphere shell with antipodal goals, m=100, T=8 s."""
    return [sphere_shell(n, seed * 100003 + i, 5.0, m=100, T=8.0)
            for i in range(n_instances)]


def poisson_schedule(rate: float, duration_s: float, seed: int = 0,
                     sizes=(8, 16, 32, 48, 64)):
    """Poisson arrival times with agent counts: list of (t_s, n, problem_seed)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        n = int(rng.choice(np.asarray(sizes)))
        out.append((t, n, seed * 1000003 + i))
        i += 1
    return out


def serving_box(n: int, problem_seed: int) -> Problem:
    """One serving request: random 8x8x4 m box, m = 100, T = 8 s."""
    return random_box(n, problem_seed, box=(8.0, 8.0, 4.0), m=100, T=8.0)


def poisson_arrivals(rate: float, duration_s: float, seed: int = 0,
                     sizes=(8, 16, 32, 48, 64)):
    """Poisson arrivals: list of (arrival_time_s, Problem) in an 8x8x4 m box."""
    return [(t, serving_box(n, ps)) for t, n, ps in
            poisson_schedule(rate, duration_s, seed, sizes)]


def stack(problems: list[Problem]):
    """Stack same-n problems into (B, n, 3) float32 start/goal arrays."""
    n = problems[0].n
    assert all(p.n == n for p in problems)
    s = np.ascontiguousarray(np.stack([p.start for p in problems]))
    g = np.ascontiguousarray(np.stack([p.goal for p in problems]))
    return s, g
