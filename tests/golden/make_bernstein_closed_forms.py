"""Writes bernstein_closed_forms.json from textbook closed forms of the
Bernstein basis of degree N on [0, 1] (no oracle code involved):

  B_{k,N}(1/2)  = C(N,k) / 2^N
  B'_{k,N}(0)   = -N if k == 0, N if k == 1, else 0
  B'_{k,N}(1)   = -N if k == N-1, N if k == N, else 0
  B''_{k,N}(0)  = N(N-1) * (1, -2, 1) for k = 0, 1, 2, else 0
  B''_{k,N}(1)  = N(N-1) * (1, -2, 1) for k = N, N-1, N-2, else 0
"""
import json
import os
from math import comb

N = 10
half = [comb(N, k) / 2 ** N for k in range(N + 1)]
d0 = [0.0] * (N + 1); d0[0] = -N; d0[1] = N
d1 = [0.0] * (N + 1); d1[N - 1] = -N; d1[N] = N
c = N * (N - 1)
dd0 = [0.0] * (N + 1); dd0[0] = c; dd0[1] = -2 * c; dd0[2] = c
dd1 = [0.0] * (N + 1); dd1[N] = c; dd1[N - 1] = -2 * c; dd1[N - 2] = c
out = {"source": "textbook closed forms of the Bernstein basis (degree 10)",
       "degree": N, "B_at_half": half, "dB_at_0": d0, "dB_at_1": d1,
       "d2B_at_0": dd0, "d2B_at_1": dd1}
with open(os.path.join(os.path.dirname(__file__), "bernstein_closed_forms.json"), "w") as f:
    json.dump(out, f, indent=1)
