// FP64 precompute of a plan, on the GPU (Sec. III-B, Eq. kkt_step_x, Remarks 1-2).
//
// Forms the Bernstein basis P, Pdot, Pddot (Eq. param), the smoothness
// Hessian block Pddot^T Pddot, the boundary rows A, the KKT matrix
//     K = [[Q_x + rho A_fc^T A_fc, A_eq^T], [A_eq, 0]]
// and its inverse from the exact agent-level closed form (two (nv + nb)-square
// inverses by Gauss-Jordan elimination with partial pivoting, one block each),
// then a self-check max |K K^-1 - I| against K assembled from its definition.
// Everything runs in float64 on the device; the host only sequences the
// launches (about 15 for a constant rho).  The iteration kernels keep the top
// n*nv rows of K^-1 in float32 (and TF32/BF16 hi/lo copies).
#include <cmath>
#include <cstdio>
#include <cstring>

#include <cuda_bf16.h>

#include "amto_internal.cuh"

namespace amto {
namespace {

__device__ double binom(int nn, int k) {
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (nn - k + i) / i;
    return c;
}

__device__ double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// Bernstein polynomial B_{k,nn}(tau); zero outside 0 <= k <= nn.
__device__ double bern(int nn, int k, double tau) {
    if (nn < 0 || k < 0 || k > nn) return 0.0;
    return binom(nn, k) * ipow(tau, k) * ipow(1.0 - tau, nn - k);
}

// P, Pdot, Pddot at t_k = k T / (m-1): derivative identities of the
// Bernstein basis, dB_{k,N} = N (B_{k-1,N-1} - B_{k,N-1}) and its second
// difference, scaled by 1/T and 1/T^2 (d/dt = (1/T) d/dtau).
__global__ void k_basis(int m, int N, double T, double* P, double* dP, double* ddP) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nv = N + 1;
    if (idx >= m * nv) return;
    int t = idx / nv, k = idx % nv;
    double tau = (double)t / (double)(m - 1);
    P[idx] = bern(N, k, tau);
    dP[idx] = N * (bern(N - 1, k - 1, tau) - bern(N - 1, k, tau)) / T;
    ddP[idx] = (double)N * (N - 1) *
               (bern(N - 2, k - 2, tau) - 2.0 * bern(N - 2, k - 1, tau) + bern(N - 2, k, tau)) /
               (T * T);
}

// PtP = P^T P, DtD = Pddot^T Pddot (nv x nv), and the boundary rows A.
__global__ void k_small(int m, int nv, unsigned mask, const double* P, const double* dP,
                        const double* ddP, double* PtP, double* DtD, double* A) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < nv * nv) {
        int k = idx / nv, l = idx % nv;
        double s1 = 0.0, s2 = 0.0;
        for (int t = 0; t < m; ++t) {
            s1 += P[t * nv + k] * P[t * nv + l];
            s2 += ddP[t * nv + k] * ddP[t * nv + l];
        }
        PtP[idx] = s1;
        DtD[idx] = s2;
    }
    if (idx < nv) {
        // rows of A in the order P_1, Pdot_1, Pddot_1, P_m, Pdot_m, Pddot_m
        const double* src[6] = {P, dP, ddP, P + (m - 1) * nv, dP + (m - 1) * nv,
                                ddP + (m - 1) * nv};
        int r = 0;
        for (int i = 0; i < 6; ++i)
            if ((mask >> i) & 1u) A[(r++) * nv + idx] = src[i][idx];
    }
}

// K of Eq. (kkt_step_x), unknowns [c (agent-major) ; multipliers (agent-major)].
// Block (i, j) of A_fc^T A_fc is the sum over pairs q of B_qi^T B_qj with
// B_qi = +P / -P for the first / second agent of pair q (Eq. A_f): every
// agent is in n-1 pairs, so the diagonal block is (n-1) P^T P, and two
// different agents share one pair with opposite signs, giving -P^T P.
// Full KKT matrix of Eq. (kkt_step_x): every agent is in n - 1 pairs and
// n_obs agent-obstacle rows (reading R-obst), so its diagonal block carries
// rho (n - 1 + n_obs) P^T P and every pair -rho P^T P off the diagonal.
__global__ void k_assemble(int n, int n_obs, int nv, int nb, double rho, const double* PtP,
                           const double* DtD, const double* A, double* K) {
    int kdim = n * (nv + nb);
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kdim * kdim) return;
    int r = (int)(idx / kdim), c = (int)(idx % kdim);
    int nvn = n * nv;
    double v = 0.0;
    if (r < nvn && c < nvn) {
        int i = r / nv, k = r % nv, j = c / nv, l = c % nv;
        v = (i == j) ? DtD[k * nv + l] + rho * (n - 1 + n_obs) * PtP[k * nv + l]
                     : -rho * PtP[k * nv + l];
    } else if (r < nvn) {
        int cc = c - nvn, j = cc / nb, rr = cc % nb, i = r / nv, k = r % nv;
        v = (i == j) ? A[rr * nv + k] : 0.0;
    } else if (c < nvn) {
        int r0 = r - nvn, i = r0 / nb, rr = r0 % nb, j = c / nv, l = c % nv;
        v = (i == j) ? A[rr * nv + l] : 0.0;
    }
    K[idx] = v;
}

// ---- Agent-level inverses (Remarks 1-2) ------------------------------------
//
// With the unknowns of agent i grouped (its nv coefficients, then its nb
// boundary multipliers), the KKT matrix of Eq. (kkt_step_x) is
//     K = I (x) K_n - 1 1^T (x) Z,   Z = [[rho P^T P, 0], [0, 0]],
// K_n = [[Pddot^T Pddot + rho (n + n_obs) P^T P, A^T], [A, 0]]: every pair
// row of Eq. (A_f) adds rho P^T P to the diagonal blocks of its two agents
// and -rho P^T P to the two off-diagonal blocks.  With 1 1^T = n Pi (Pi the
// projector on the agents' mean), K = (I - Pi) (x) K_n + Pi (x) K_0 where
// K_0 = K_n - n Z carries rho n_obs P^T P (0 without obstacles: the
// smoothness-only matrix of the initial solve), so
//     K^-1 = I (x) K_n^-1 + (1/n) 1 1^T (x) (K_0^-1 - K_n^-1)
// exactly.  Only the two (nv + nb)-square agent-level matrices are inverted.

constexpr int kMaxAgentDim = 32;  // nv + nb <= 16 + 6

// One block per agent-level matrix [[DtD + w PtP, A^T], [A, 0]] (weights w in
// `wts`): assembled into shared memory as [M | I] and inverted by
// Gauss-Jordan elimination with partial pivoting (largest |pivot|, ties to
// the smallest row), FP64.  A zero pivot sets *singular.
__global__ void k_agent_inverse(int nv, int nb, const double* DtD, const double* PtP,
                                const double* A, const double* wts, double* inv,
                                int* singular) {
    __shared__ double W[kMaxAgentDim][2 * kMaxAgentDim + 1];
    __shared__ int s_piv;
    const int d = nv + nb, tid = threadIdx.x, nt = blockDim.x;
    const double w = wts[blockIdx.x];
    for (int e = tid; e < d * 2 * d; e += nt) {
        const int r = e / (2 * d), c = e % (2 * d);
        double v;
        if (c >= d) v = (c - d == r) ? 1.0 : 0.0;
        else if (r < nv && c < nv) v = DtD[r * nv + c] + w * PtP[r * nv + c];
        else if (r < nv) v = A[(c - nv) * nv + r];
        else if (c < nv) v = A[(r - nv) * nv + c];
        else v = 0.0;
        W[r][c] = v;
    }
    __syncthreads();
    for (int c = 0; c < d; ++c) {
        if (tid == 0) {
            int p = c;
            double best = fabs(W[c][c]);
            for (int r = c + 1; r < d; ++r)
                if (fabs(W[r][c]) > best) { best = fabs(W[r][c]); p = r; }
            if (!(best > 0.0)) *singular = 1;
            s_piv = p;
        }
        __syncthreads();
        const int p = s_piv;
        const double pv = W[p][c];
        if (!(fabs(pv) > 0.0)) return;  // uniform over the block
        __syncthreads();
        for (int j = tid; j < 2 * d; j += nt) {  // swap rows c and p, scale row c
            const double a = W[c][j], b = W[p][j];
            if (p != c) W[p][j] = a;
            W[c][j] = b / pv;
        }
        __syncthreads();
        // eliminate column c from the other rows; column c is read as the
        // multiplier and left as is (never read again)
        for (int e = tid; e < d * (2 * d - c - 1); e += nt) {
            const int r = e / (2 * d - c - 1), j = c + 1 + e % (2 * d - c - 1);
            if (r == c) continue;
            const double f = W[r][c];
            if (f != 0.0) W[r][j] -= f * W[c][j];
        }
        __syncthreads();
    }
    double* out = inv + (size_t)blockIdx.x * d * d;
    for (int e = tid; e < d * d; e += nt) out[e] = W[e / d][d + e % d];
}

// Dense K^-1 (kdim x kdim, unknowns [all coefficients ; all multipliers],
// each agent-major) from the agent-level inverses by the closed form above.
__global__ void k_kron_inverse(int n, int nv, int nb, const double* Kn_inv, const double* K0_inv,
                               double* Kinv) {
    const int d = nv + nb, nvn = n * nv, kdim = n * d;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kdim * kdim) return;
    const int r = (int)(idx / kdim), c = (int)(idx % kdim);
    const int i = r < nvn ? r / nv : (r - nvn) / nb, q = r < nvn ? r % nv : nv + (r - nvn) % nb;
    const int j = c < nvn ? c / nv : (c - nvn) / nb, q2 = c < nvn ? c % nv : nv + (c - nvn) % nb;
    const double kn = Kn_inv[q * d + q2];
    const double mean = (K0_inv[q * d + q2] - kn) / (double)n;
    Kinv[idx] = i == j ? kn + mean : mean;
}

// max |K K^-1 - I| as the bits of a non-negative double (atomicMax on the
// integer pattern orders non-negative doubles correctly).
__global__ void k_check(int N, const double* K, const double* Kinv, unsigned long long* err) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    int r = (int)(idx / N), c = (int)(idx % N);
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += K[(long long)r * N + k] * Kinv[(long long)k * N + c];
    double e = fabs(s - (r == c ? 1.0 : 0.0));
    if (!(e == e)) e = INFINITY;
    atomicMax(err, (unsigned long long)__double_as_longlong(e));
}

__global__ void k_to_f32(long long count, const double* src, float* dst) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < count) dst[idx] = (float)src[idx];
}

// The rounding error of k_to_f32: lo = float32(x - float32(x)), so that
// (hi, lo) carries x to about 2^-48 relative.
__global__ void k_to_f32_lo(long long count, const double* src, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < count) lo[idx] = (float)(src[idx] - (double)(float)src[idx]);
}

// Round a float32 to TF32 (10 explicit mantissa bits), to nearest, ties to even.
__device__ __forceinline__ float tf32_round(float x) {
    unsigned u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0xfffu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xffffe000u);
}

// Split the top rows of K^-1 for the tensor-core apply: hi = TF32(K^-1),
// lo = float32(K^-1 - hi), rows padded to ld columns.
__global__ void k_split_top(int rows, int kdim, int ld, const double* Kinv, float* hi, float* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * ld) return;
    int r = (int)(idx / ld), c = (int)(idx % ld);
    double x = (c < kdim) ? Kinv[(long long)r * kdim + c] : 0.0;
    float h = tf32_round((float)x);
    hi[idx] = h;
    lo[idx] = (float)(x - (double)h);
}

// BF16 split of the top rows of K^-1: hi = BF16(K^-1), lo = BF16(K^-1 - hi).
__global__ void k_split_top_bf16(int rows, int kdim, int ld, const double* Kinv,
                                 __nv_bfloat16* hi, __nv_bfloat16* lo) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)rows * ld) return;
    int r = (int)(idx / ld), c = (int)(idx % ld);
    double x = (c < kdim) ? Kinv[(long long)r * kdim + c] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
}

// Rows [0, nv) of an agent-level inverse as float32 [nv][nv + nb].
__global__ void k_agent_top(int nv, int nb, const double* Kinv, float* out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nv * (nv + nb)) return;
    out[idx] = (float)Kinv[idx];
}

// E0 = rows [0, nv) and columns [nv, nv+nb) of the agent-level inverse.
__global__ void k_extract_e0(int nv, int nb, const double* K0inv, float* E0) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nv * nb) return;
    int k = idx / nb, r = idx % nb;
    E0[idx] = (float)K0inv[k * (nv + nb) + nv + r];
}

inline unsigned blocks(long long count, int threads) {
    return (unsigned)((count + threads - 1) / threads);
}

}  // namespace

amto_status precompute(amto_plan_s* pl) {
    const int m = pl->m, N = pl->N, nv = pl->nv, nb = pl->nb, n = pl->n, kdim = pl->kdim;
    const int d = nv + nb, J = pl->sched.J, n_obs = pl->prm.n_obstacles;
    cudaStream_t s = pl->cap_stream;
    if (d > kMaxAgentDim) {
        set_error("agent-level KKT block larger than supported");
        return AMTO_EINVAL;
    }
    // agent-level matrices: [0] smoothness only (w = 0); per stage j the
    // relative block K_n (w = rho_j (n + n_obs)) and, with obstacles, the
    // common block K_0 (w = rho_j n_obs)
    const int per_stage = n_obs > 0 ? 2 : 1, nmat = 1 + J * per_stage;
    double wts[1 + 2 * kMaxRhoStages];
    wts[0] = 0.0;
    for (int j = 0; j < J; ++j) {
        wts[1 + j * per_stage] = pl->sched.rho_d[j] * (n + n_obs);
        if (n_obs > 0) wts[2 + j * per_stage] = pl->sched.rho_d[j] * n_obs;
    }
    double *P = nullptr, *dP = nullptr, *ddP = nullptr, *PtP = nullptr, *DtD = nullptr,
           *A = nullptr, *K = nullptr, *Ainv = nullptr, *dw = nullptr;
    int* si = nullptr;
    unsigned long long* err = nullptr;
    amto_status st = AMTO_OK;

#define PC_ALLOC(ptr, bytes)                                                        \
    if (st == AMTO_OK && cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {      \
        cudaGetLastError();                                                         \
        set_error("cudaMalloc failed in precompute");                               \
        st = AMTO_ENOMEM;                                                           \
    }
    PC_ALLOC(P, sizeof(double) * m * nv);
    PC_ALLOC(dP, sizeof(double) * m * nv);
    PC_ALLOC(ddP, sizeof(double) * m * nv);
    PC_ALLOC(PtP, sizeof(double) * nv * nv);
    PC_ALLOC(DtD, sizeof(double) * nv * nv);
    PC_ALLOC(A, sizeof(double) * nb * nv);
    PC_ALLOC(K, sizeof(double) * (size_t)kdim * kdim);
    PC_ALLOC(Ainv, sizeof(double) * nmat * d * d);
    PC_ALLOC(dw, sizeof(double) * nmat);
    PC_ALLOC(si, sizeof(int));
    PC_ALLOC(err, sizeof(unsigned long long) * J);
#undef PC_ALLOC

    if (st == AMTO_OK &&
        (cudaMemcpyAsync(dw, wts, sizeof(double) * nmat, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemsetAsync(si, 0, sizeof(int), s) != cudaSuccess ||
         cudaMemsetAsync(err, 0, sizeof(unsigned long long) * J, s) != cudaSuccess)) {
        cudaGetLastError();
        set_error("precompute: copy of the agent-level weights failed");
        st = AMTO_ECUDA;
    }
    if (st == AMTO_OK) {
        k_basis<<<blocks(m * nv, 128), 128, 0, s>>>(m, N, pl->prm.T, P, dP, ddP);
        k_small<<<blocks(nv * nv, 128), 128, 0, s>>>(m, nv, pl->prm.bc_mask, P, dP, ddP, PtP,
                                                      DtD, A);
        k_agent_inverse<<<nmat, 128, 0, s>>>(nv, nb, DtD, PtP, A, dw, Ainv, si);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("precompute kernel launch failed");
            st = AMTO_ECUDA;
        }
    }
    const double* K0inv = Ainv;  // smoothness-only block
    // one cached inverse per rho stage (Remarks 1-2: K depends on rho and n
    // only); the last one formed, stage 0, stays in Kinv64
    const int rows = n * nv;
    for (int j = J - 1; j >= 0 && st == AMTO_OK; --j) {
        const double* Kninv = Ainv + (size_t)(1 + j * per_stage) * d * d;
        const double* Kcinv = n_obs > 0 ? Ainv + (size_t)(2 + j * per_stage) * d * d : K0inv;
        k_kron_inverse<<<blocks((long long)kdim * kdim, 256), 256, 0, s>>>(n, nv, nb, Kninv, Kcinv,
                                                                           pl->Kinv64);
        // self-check against K assembled directly from its definition
        k_assemble<<<blocks((long long)kdim * kdim, 256), 256, 0, s>>>(n, n_obs, nv, nb,
                                                                       pl->sched.rho_d[j], PtP,
                                                                       DtD, A, K);
        k_check<<<blocks((long long)kdim * kdim, 256), 256, 0, s>>>(kdim, K, pl->Kinv64, err + j);
        // top n*nv rows of the row-major inverse are its first rows*kdim entries
        k_to_f32<<<blocks((long long)rows * kdim, 256), 256, 0, s>>>(
            (long long)rows * kdim, pl->Kinv64, pl->Ktop + j * pl->ks_top);
        if (pl->Kt_hi)
            k_split_top<<<blocks((long long)rows * pl->kp, 256), 256, 0, s>>>(
                rows, kdim, pl->kp, pl->Kinv64, pl->Kt_hi + j * pl->ks_tc,
                pl->Kt_lo + j * pl->ks_tc);
        if (pl->Kb_hi)
            k_split_top_bf16<<<blocks((long long)rows * pl->kp8, 256), 256, 0, s>>>(
                rows, kdim, pl->kp8, pl->Kinv64,
                reinterpret_cast<__nv_bfloat16*>(pl->Kb_hi) + j * pl->ks_bf,
                reinterpret_cast<__nv_bfloat16*>(pl->Kb_lo) + j * pl->ks_bf);
        k_agent_top<<<blocks(nv * d, 64), 64, 0, s>>>(nv, nb, Kninv, pl->Kag + j * pl->ks_ag);
        k_agent_top<<<blocks(nv * d, 64), 64, 0, s>>>(nv, nb, Kcinv,
                                                      pl->Kag + j * pl->ks_ag + nv * d);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("precompute kernel launch failed");
            st = AMTO_ECUDA;
        }
    }
    if (st == AMTO_OK) {
        k_extract_e0<<<blocks(nv * nb, 64), 64, 0, s>>>(nv, nb, K0inv, pl->E0);
        k_to_f32<<<blocks(m * nv, 128), 128, 0, s>>>((long long)m * nv, P, pl->P32);
        k_to_f32_lo<<<blocks(m * nv, 128), 128, 0, s>>>((long long)m * nv, P, pl->P32lo);
        k_to_f32<<<blocks(nv * nv, 128), 128, 0, s>>>((long long)nv * nv, DtD, pl->Q32);
        k_to_f32<<<blocks(nb * nv, 128), 128, 0, s>>>((long long)nb * nv, A, pl->A32);
        cudaMemcpyAsync(pl->P64, P, sizeof(double) * m * nv, cudaMemcpyDeviceToDevice, s);
    }
    int singular = 0;
    unsigned long long bits[kMaxRhoStages] = {};
    if (st == AMTO_OK &&
        (cudaMemcpyAsync(&singular, si, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(bits, err, sizeof(unsigned long long) * J, cudaMemcpyDeviceToHost, s) !=
             cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)) {
        set_error("precompute failed to run");
        st = AMTO_ECUDA;
    }
    if (st == AMTO_OK && singular) {
        set_error("KKT matrix is singular (zero pivot in an agent-level inverse)");
        st = AMTO_ENUMERIC;
    }
    double worst = 0.0;
    for (int j = 0; j < J && st == AMTO_OK; ++j) {
        double e;
        memcpy(&e, &bits[j], sizeof(e));
        worst = e > worst ? e : worst;
        if (!(e < 1e-6)) {
            char buf[160];
            snprintf(buf, sizeof(buf), "KKT inverse self-check failed: max|K K^-1 - I| = %g", e);
            set_error(buf);
            st = AMTO_ENUMERIC;
        }
    }
    pl->kkt_check = worst;
    cudaFree(P); cudaFree(dP); cudaFree(ddP); cudaFree(PtP); cudaFree(DtD); cudaFree(A);
    cudaFree(K); cudaFree(Ainv); cudaFree(dw); cudaFree(si); cudaFree(err);
    return st;
}

}  // namespace amto
