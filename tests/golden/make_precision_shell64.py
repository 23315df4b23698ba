"""Writes precision_shell64.npz: the FP64 oracle's trajectory coefficients
xi^k of sampled instances of the batched 64-agent sphere-shell workload
(lambda-free projection, reading R3), for the per-precision error report.

Calls only the oracle (Algorithm 1 in FP64) and the seeded input generator.
Stored per sample i and k in KS: xi^k (3 x n x (N+1)), plus the oracle's own
sensitivity horizon K_par of each sample: the largest iteration count k such
that, for every iteration up to k, runs started from inputs perturbed by
relative noise of 1e-7 stay within 1e-4 (relative, max norm) of the
unperturbed run.  Past K_par the problem itself amplifies rounding noise
beyond 1e-4, so an error against the oracle there measures the problem's
chaos, not the arithmetic.

    python tests/golden/make_precision_shell64.py      (about a minute on 8 cores)
"""
import multiprocessing as mp
import os
import sys

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")   # one BLAS thread per pool worker

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KS = (1, 2, 5, 10, 20, 200)
SAMPLES = (0, 85, 170, 255)   # instance indices of the 256-instance batch (seed 0)
N_AGENTS = 64
DRAWS = 2                     # perturbed runs per sample
NOISE = 1e-7
DIVERGE = 1e-4


def _run(task):
    """One oracle solve of max(KS) iterations; returns xi at every iteration."""
    import oracle as O
    import workloads as W
    sample, draw = task
    p = W.shell_batch(sample + 1, seed=0, n=N_AGENTS)[sample]
    start = p.start.astype(np.float64)
    goal = p.goal.astype(np.float64)
    if draw >= 0:
        rng = np.random.default_rng(1000 * sample + draw)
        start = start * (1 + NOISE * rng.standard_normal(start.shape))
        goal = goal * (1 + NOISE * rng.standard_normal(goal.shape))
    M = O.build_matrices(p.n, p.m, p.degree, p.T, p.a, p.b, p.rho)
    beq = O.boundary_values(start, goal)
    st = O.init_state(M, beq, "R3")
    xs = np.empty((max(KS),) + st.xi.shape)
    for k in range(max(KS)):
        st = O.am_iteration(M, st, beq, "R3")
        xs[k] = st.xi
    return sample, draw, xs, float(st.r_max)


def main():
    tasks = [(s, -1) for s in SAMPLES] + [(s, d) for s in SAMPLES for d in range(DRAWS)]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        res = pool.map(_run, tasks)
    base = {s: (xs, r) for s, d, xs, r in res if d < 0}
    kpar = {}
    for s, d, xs, _ in res:
        if d < 0:
            continue
        ref = base[s][0]
        div = np.abs(xs - ref).reshape(len(xs), -1).max(1) / np.abs(ref).reshape(len(ref), -1).max(1)
        bad = np.nonzero(div > DIVERGE)[0]
        k = int(bad[0]) if len(bad) else max(KS)   # iterations 1..k stay within DIVERGE
        kpar[s] = min(kpar.get(s, max(KS)), k)
    out = {"ks": np.array(KS), "samples": np.array(SAMPLES),
           "k_par": np.array([kpar[s] for s in SAMPLES]),
           "r_max_final": np.array([base[s][1] for s in SAMPLES])}
    for s in SAMPLES:
        for k in KS:
            out[f"xi_s{s}_k{k}"] = base[s][0][k - 1]
    np.savez_compressed(os.path.join(HERE, "precision_shell64.npz"), **out)
    print("K_par per sample:", dict(zip(SAMPLES, out["k_par"].tolist())))


if __name__ == "__main__":
    main()
