// FP64 precompute of a plan, on the GPU (Sec. III-B, Eq. kkt_step_x, Remarks 1-2).
//
// Forms the Bernstein basis P, Pdot, Pddot (Eq. param), the smoothness
// Hessian block Pddot^T Pddot, the boundary rows A, the KKT matrix
//     K = [[Q_x + rho A_fc^T A_fc, A_eq^T], [A_eq, 0]]
// and its inverse by Gauss-Jordan elimination with partial pivoting, then a
// self-check max |K K^-1 - I|.  Everything runs in float64 on the device;
// the host only sequences the launches.  The iteration kernels keep the top
// n*nv rows of K^-1 in float32.
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

// Agent-level KKT matrix [[Pddot^T Pddot, A^T], [A, 0]] of the
// smoothness-only initial solve.
// Agent-level KKT matrix [[DtD + w PtP, A^T], [A, 0]] (w = 0: smoothness only,
// the ring of all agents moving together; w = rho n: the block of one agent
// relative to the others, Remark 1's structure of the full matrix).
__global__ void k_assemble_agent(int nv, int nb, const double* DtD, const double* PtP, double w,
                                 const double* A, double* K) {
    int d = nv + nb;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= d * d) return;
    int r = idx / d, c = idx % d;
    double v = 0.0;
    if (r < nv && c < nv) v = DtD[r * nv + c] + w * PtP[r * nv + c];
    else if (r < nv) v = A[(c - nv) * nv + r];
    else if (c < nv) v = A[(r - nv) * nv + c];
    K[idx] = v;
}

// ---- Gauss-Jordan with partial pivoting on W = [K | I] (N x 2N) ----------

__global__ void k_gj_init(int N, const double* K, double* W) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2LL * N * N) return;
    int r = (int)(idx / (2 * N)), c = (int)(idx % (2 * N));
    W[idx] = (c < N) ? K[(long long)r * N + c] : (c - N == r ? 1.0 : 0.0);
}

// Pivot row p = argmax_{r >= c} |W[r][c]| (ties: smallest r); pv = W[p][c].
__global__ void k_gj_pivot(int N, int c, const double* W, int* piv, double* pv, int* singular) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
    double best = -1.0;
    int bi = N;
    for (int r = c + threadIdx.x; r < N; r += blockDim.x) {
        double v = fabs(W[(long long)r * 2 * N + c]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v2 = sv[threadIdx.x + s];
            int i2 = si[threadIdx.x + s];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int p = si[0];
        *piv = p;
        double v = (p < N) ? W[(long long)p * 2 * N + c] : 0.0;
        *pv = v;
        if (!(fabs(v) > 0.0)) *singular = 1;
    }
}

// Swap rows c and piv, divide the new row c by the pivot value.
__global__ void k_gj_swap_scale(int N, int c, double* W, const int* piv, const double* pv) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2 * N) return;
    int p = *piv;
    double v = *pv;
    if (!(fabs(v) > 0.0) || p >= N) return;
    double* rc = W + (long long)c * 2 * N;
    double* rp = W + (long long)p * 2 * N;
    double a = rc[j], b = rp[j];
    if (p != c) rp[j] = a;
    rc[j] = b / v;
}

// Eliminate column c from every other row.  Only columns j > c of the left
// half and the whole right half change; column c itself is left as is (it is
// never read again), so W[r][c] is a stable multiplier during this launch.
__global__ void k_gj_elim(int N, int c, double* W, const double* pv) {
    if (!(fabs(*pv) > 0.0)) return;
    int width = (N - c - 1) + N;
    int jj = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (jj >= width || r == c) return;
    int j = (jj < N - c - 1) ? (c + 1 + jj) : (N + (jj - (N - c - 1)));
    double* wr = W + (long long)r * 2 * N;
    double f = wr[c];
    if (f != 0.0) wr[j] -= f * W[(long long)c * 2 * N + j];
}

__global__ void k_gj_extract(int N, const double* W, double* Kinv) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    int r = (int)(idx / N), c = (int)(idx % N);
    Kinv[idx] = W[(long long)r * 2 * N + N + c];
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

// Gauss-Jordan inverse of the N x N device matrix K into Kinv (W: N x 2N).
amto_status invert(int N, const double* K, double* Kinv, double* W, int* scratch_i,
                   double* scratch_d, cudaStream_t s) {
    k_gj_init<<<blocks(2LL * N * N, 256), 256, 0, s>>>(N, K, W);
    AMTO_CUDA_TRY(cudaMemsetAsync(scratch_i + 1, 0, sizeof(int), s));
    for (int c = 0; c < N; ++c) {
        k_gj_pivot<<<1, 1024, 0, s>>>(N, c, W, scratch_i, scratch_d, scratch_i + 1);
        k_gj_swap_scale<<<blocks(2 * N, 256), 256, 0, s>>>(N, c, W, scratch_i, scratch_d);
        int width = (N - c - 1) + N;
        dim3 g(blocks(width, 256), N);
        k_gj_elim<<<g, 256, 0, s>>>(N, c, W, scratch_d);
    }
    k_gj_extract<<<blocks((long long)N * N, 256), 256, 0, s>>>(N, W, Kinv);
    AMTO_CUDA_TRY(cudaGetLastError());
    int singular = 0;
    AMTO_CUDA_TRY(cudaMemcpyAsync(&singular, scratch_i + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMTO_CUDA_TRY(cudaStreamSynchronize(s));
    if (singular) {
        set_error("KKT matrix is singular (zero pivot in Gauss-Jordan elimination)");
        return AMTO_ENUMERIC;
    }
    return AMTO_OK;
}

}  // namespace

amto_status precompute(amto_plan_s* pl) {
    const int m = pl->m, N = pl->N, nv = pl->nv, nb = pl->nb, n = pl->n, kdim = pl->kdim;
    cudaStream_t s = pl->cap_stream;
    double *P = nullptr, *dP = nullptr, *ddP = nullptr, *PtP = nullptr, *DtD = nullptr,
           *A = nullptr, *K = nullptr, *W = nullptr, *K0 = nullptr, *K0inv = nullptr,
           *Kn = nullptr, *Kninv = nullptr, *Ko = nullptr, *Koinv = nullptr, *sd = nullptr;
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
    PC_ALLOC(W, sizeof(double) * (size_t)kdim * kdim * 2);
    PC_ALLOC(K0, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(K0inv, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(Kn, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(Kninv, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(Ko, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(Koinv, sizeof(double) * (nv + nb) * (nv + nb));
    PC_ALLOC(sd, sizeof(double) * 4);
    PC_ALLOC(si, sizeof(int) * 4);
    PC_ALLOC(err, sizeof(unsigned long long));
#undef PC_ALLOC

    if (st == AMTO_OK) {
        k_basis<<<blocks(m * nv, 128), 128, 0, s>>>(m, N, pl->prm.T, P, dP, ddP);
        k_small<<<blocks(nv * nv, 128), 128, 0, s>>>(m, nv, pl->prm.bc_mask, P, dP, ddP, PtP,
                                                      DtD, A);
        k_assemble_agent<<<blocks((nv + nb) * (nv + nb), 128), 128, 0, s>>>(nv, nb, DtD, PtP, 0.0,
                                                                           A, K0);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("precompute kernel launch failed");
            st = AMTO_ECUDA;
        }
    }
    if (st == AMTO_OK) st = invert(nv + nb, K0, K0inv, W, si, sd, s);
    // one cached inverse per rho stage (Remarks 1-2: K depends on rho and n
    // only); the last one computed, stage 0, stays in Kinv64
    const int rows = n * nv, d = nv + nb;
    double worst = 0.0;
    for (int j = pl->sched.J - 1; j >= 0 && st == AMTO_OK; --j) {
        const double rho = pl->sched.rho_d[j];
        const int n_obs = pl->prm.n_obstacles;
        k_assemble<<<blocks((long long)kdim * kdim, 256), 256, 0, s>>>(n, n_obs, nv, nb, rho, PtP,
                                                                       DtD, A, K);
        // agent-level blocks of the structured inverse: the relative motion
        // sees rho (n + n_obs) P^T P, the common motion rho n_obs P^T P
        k_assemble_agent<<<blocks(d * d, 128), 128, 0, s>>>(nv, nb, DtD, PtP, rho * (n + n_obs), A,
                                                            Kn);
        if (n_obs > 0)
            k_assemble_agent<<<blocks(d * d, 128), 128, 0, s>>>(nv, nb, DtD, PtP, rho * n_obs, A,
                                                                Ko);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("precompute kernel launch failed");
            st = AMTO_ECUDA;
            break;
        }
        st = invert(nv + nb, Kn, Kninv, W, si, sd, s);
        if (st == AMTO_OK && n_obs > 0) st = invert(nv + nb, Ko, Koinv, W, si, sd, s);
        if (st == AMTO_OK) st = invert(kdim, K, pl->Kinv64, W, si, sd, s);
        if (st != AMTO_OK) break;
        cudaMemsetAsync(err, 0, sizeof(unsigned long long), s);
        k_check<<<blocks((long long)kdim * kdim, 256), 256, 0, s>>>(kdim, K, pl->Kinv64, err);
        unsigned long long bits = 0;
        cudaMemcpyAsync(&bits, err, sizeof(bits), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("precompute self-check failed to run");
            st = AMTO_ECUDA;
            break;
        }
        double e;
        memcpy(&e, &bits, sizeof(e));
        worst = e > worst ? e : worst;
        if (!(e < 1e-6)) {
            char buf[160];
            snprintf(buf, sizeof(buf), "KKT inverse self-check failed: max|K K^-1 - I| = %g", e);
            set_error(buf);
            st = AMTO_ENUMERIC;
            break;
        }
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
        k_agent_top<<<blocks(nv * d, 64), 64, 0, s>>>(nv, nb, n_obs > 0 ? Koinv : K0inv,
                                                      pl->Kag + j * pl->ks_ag + nv * d);
    }
    pl->kkt_check = worst;
    if (st == AMTO_OK) {
        k_extract_e0<<<blocks(nv * nb, 64), 64, 0, s>>>(nv, nb, K0inv, pl->E0);
        k_to_f32<<<blocks(m * nv, 128), 128, 0, s>>>((long long)m * nv, P, pl->P32);
        k_to_f32<<<blocks(nv * nv, 128), 128, 0, s>>>((long long)nv * nv, DtD, pl->Q32);
        k_to_f32<<<blocks(nb * nv, 128), 128, 0, s>>>((long long)nb * nv, A, pl->A32);
        cudaMemcpyAsync(pl->P64, P, sizeof(double) * m * nv, cudaMemcpyDeviceToDevice, s);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            set_error("precompute extraction failed");
            st = AMTO_ECUDA;
        }
    }
    cudaFree(P); cudaFree(dP); cudaFree(ddP); cudaFree(PtP); cudaFree(DtD); cudaFree(A);
    cudaFree(K); cudaFree(W); cudaFree(K0); cudaFree(K0inv); cudaFree(Kn); cudaFree(Kninv);
    cudaFree(Ko); cudaFree(Koinv); cudaFree(sd); cudaFree(si);
    cudaFree(err);
    return st;
}

}  // namespace amto
