"""The stored FP64 reference of the per-precision error report
(tests/golden/precision_shell64.npz) is the oracle's output on the seeded
sphere-shell inputs: its first two iterates of one sample are recomputed
here with the oracle (Algorithm 1, reading R3) and must agree to rounding."""
import os

import numpy as np

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "precision_shell64.npz")


def test_stored_reference_is_the_oracle_on_the_seeded_inputs():
    z = np.load(GOLD)
    assert list(z["ks"]) == [1, 2, 5, 10, 20, 200]
    assert list(z["samples"]) == [0, 85, 170, 255]
    assert np.all((z["k_par"] >= 1) & (z["k_par"] <= 200))
    p = W.shell_batch(1, seed=0, n=64)[0]
    M = O.build_matrices(p.n, p.m, p.degree, p.T, p.a, p.b, p.rho)
    beq = O.boundary_values(p.start.astype(np.float64), p.goal.astype(np.float64))
    st = O.init_state(M, beq, "R3")
    for k in (1, 2):
        st = O.am_iteration(M, st, beq, "R3")
        ref = z[f"xi_s0_k{k}"]
        assert ref.shape == st.xi.shape
        assert np.abs(st.xi - ref).max() <= 1e-9 * np.abs(ref).max()
