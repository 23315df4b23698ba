// Structured application of the cached KKT inverse (AMTO_APPLY_KRONECKER),
// shared by the batched kernels and the one-block-per-instance solver.
#pragma once

#include "amto_internal.cuh"

namespace amto {

// One axis of one instance by one block (all threads call it):
// K^-1 = I (x) K_n^-1 + (1/n) 1 1^T (x) (K_0^-1 - K_n^-1) in the agent-major
// order, so xi_i += K_n^-1_top (r_i - r_mean) + K_0^-1_top r_mean with r_i the
// 17-vector [g_i; e_i] of agent i.  Kag holds the two top blocks [2][nv][nv+nb].
__device__ __forceinline__ void kron_apply_axis(const float* r, int n, int nv, int nb,
                                                const float* Kag, float* x, float* sm) {
    const int d = nv + nb, nvn = n * nv, tid = threadIdx.x, bd = blockDim.x;
    float* rbar = sm;       // [d]
    float* z = sm + d;      // [nv]  K_0^-1_top rbar
    // mean over agents: one warp per component, lanes over agents, a fixed
    // shuffle tree
    const int warp = tid >> 5, lane = tid & 31, nw = bd >> 5;
    for (int c = warp; c < d; c += nw) {
        float acc = 0.f;
        if (c < nv)
            for (int i = lane; i < n; i += 32) acc += r[i * nv + c];
        else
            for (int i = lane; i < n; i += 32) acc += r[nvn + i * nb + (c - nv)];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) rbar[c] = acc / (float)n;
    }
    __syncthreads();
    const float* K0 = Kag + nv * d;
    for (int k = tid; k < nv; k += bd) {
        float acc = 0.f;
        for (int c = 0; c < d; ++c) acc = fmaf(K0[k * d + c], rbar[c], acc);
        z[k] = acc;
    }
    __syncthreads();
    for (int o = tid; o < nvn; o += bd) {
        const int i = o / nv, k = o % nv;
        const float* kr = Kag + k * d;
        float acc = z[k];
        for (int c = 0; c < nv; ++c) acc = fmaf(kr[c], r[i * nv + c] - rbar[c], acc);
        for (int c = 0; c < nb; ++c)
            acc = fmaf(kr[nv + c], r[nvn + i * nb + c] - rbar[nv + c], acc);
        x[o] += acc;
    }
}

}  // namespace amto
