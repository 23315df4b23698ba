// Final residual of the lambda-free reading, in FP64 (Algorithm 1's r_max at
// the last iterate; reading R-lambda: f_c = Delta min(0, 1 - 1/s), so
// ||f_c|| = |Delta| (1/s - 1) inside the spheroid and exactly 0 outside).
//
// Three steps, none of which evaluates every pair-time in FP64 (the FP64 rate
// of this part is about 1/64 of its float32 rate):
//
//  1. Unit skip.  The last pair pass left, per (instance, time chunk) unit,
//     its float32 maximum of ||f_c|| (rpart) and its smallest s^2 (spart).
//     The float32 positions of that pass are within 12.1 u C of the exact ones
//     (u = 2^-24, C = the instance's largest |coefficient|: the Bernstein
//     basis is a non-negative partition of unity), and ||f_c|| is Lipschitz in
//     Delta with constant 1 + kappa / |Delta| (kappa bounds the derivative of
//     the spheroid radius along a direction), where |Delta| >= l_min s.  That
//     bounds each unit's true maximum within [rt - slack, rt + slack]; a unit
//     whose upper bound is below the largest lower bound of the instance
//     cannot hold the maximum and is skipped.
//  2. Screen (k_final_screen, one block per remaining unit).  Positions as
//     float pairs (hi + lo, within about 1e-13 C of the FP64 positions) from
//     the basis as a float pair and the float32 coefficients, by error-free
//     products and compensated sums; Delta formed from them keeps its
//     direction even for nearly coincident agents.  Agent pairs whose boxes
//     over the unit's samples stay apart, and pair-times whose hi parts
//     already put them outside, have f_c = 0 exactly; every other pair-time
//     gets a float32 value within a stated bound of its true value.  Each
//     unit keeps its maximum and the pair-times that can reach it.
//  3. Confirm (k_final_confirm, one block per instance).  The pair-times that
//     can reach the instance's screened maximum are recomputed in FP64
//     (positions from the FP64 basis and the float32 coefficients); their
//     maximum is the reported residual.  A unit with more such pair-times
//     than its list holds is screened again by this block with the
//     instance's threshold.
#include <cfloat>
#include <cmath>

#include "amto_internal.cuh"
#include "pair_math.cuh"

namespace amto {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kU = 5.9604645e-8f;       // 2^-24, the float32 unit roundoff

// Error-free transformations (Knuth's two-sum; the product's rounding error
// recovered by a fused multiply-add), written with explicit roundings so the
// compiler cannot contract or reassociate them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

struct FreeArgs {
    const int* list;     // instances (NULL: 0..grid-1)
    int n, m, nv, n_chunks, TC, npad;
    int TS, NS;          // samples per screening chunk (a divisor of TC), chunks per instance
    int skip;            // rpart / spart of the last pair pass are valid
    float out_rel;       // 8 * 2^-23 / l_min: the quick outside test's margin per unit of C
    float wxy_h, wxy_l, wz_h, wz_l;  // 1/l_xy^2 and 1/l_z^2 as float pairs
    float lz;            // l_z (the degenerate direction's length, reading R-degen)
    float lmin, lmax, kappa;
    double ia2, ib2;
    const float* xi;
    const float* P32;    // float32(P64)
    const float* P32lo;  // float32(P64 - P32)
    const double* P64;
    const int* flags;
    const float* rpart;
    const float* spart;
    float* fin;          // [B][NS][kFinRecFloats]
    int* work;           // [B NS] screening chunks to do, b NS + s
    unsigned* wctl;      // [0] chunks listed, [1] chunks taken (cleared before the plan kernel)
    float* olim;         // [B] the quick outside test's limit per instance
    unsigned long long* r64;
    int n_obs;
    const float* obst;   // [B][n_obs][5]
};

// Shared memory of a screening block (floats): positions hi and lo as float4
// (x, y, z, 0) [npad][TC], obstacles (centre, weights as float pairs, l_z),
// each agent's box over the unit's samples (hi parts) [2][3][npad], the
// instance's coefficients [3][npad][nv], the unit's basis rows hi and lo
// [TC][nv], and a list of kPairBatch agent pairs (two bytes each).
constexpr int kObstF = 8;
constexpr int kPairBatch = 2048;
__host__ __device__ inline size_t free_smem_floats(int TC, int npad, int n_obs, int nv) {
    return (size_t)2 * 4 * npad * TC + (size_t)kObstF * n_obs + (size_t)6 * npad +
           (size_t)3 * npad * nv + (size_t)2 * TC * nv + kPairBatch / 2;
}
struct FreeSmem {
    float4 *Xh, *Xl;
    float *Os, *Bx, *Cf, *Ph, *Pl;
    unsigned short* list;
    __device__ FreeSmem(float* base, int TC, int npad, int n_obs, int nv) {
        Xh = reinterpret_cast<float4*>(base);
        Xl = Xh + (size_t)npad * TC;
        Os = reinterpret_cast<float*>(Xl + (size_t)npad * TC);
        Bx = Os + (size_t)kObstF * n_obs;
        Cf = Bx + (size_t)6 * npad;
        Ph = Cf + (size_t)3 * npad * nv;
        Pl = Ph + (size_t)TC * nv;
        list = reinterpret_cast<unsigned short*>(Pl + (size_t)TC * nv);
    }
};

// Quick test on the hi parts: true when the pair-time is certainly outside
// the spheroid (f_c = 0 exactly).  Each hi part is within 2^-24 C of its
// position, so their difference is within 2^-23 C (+ its own rounding) of
// Delta on each axis, and near s = 1 (where |Delta| >= l_min) s^2 is off by
// at most 2 sqrt(3) 2^-23 C / l_min; out_lim = 1 + 1e-5 + twice that.
__device__ __forceinline__ bool quick_outside(const float4& hi, const float4& hj, float wxy_h,
                                             float wz_h, float out_lim) {
    const float qx = hi.x - hj.x, qy = hi.y - hj.y, qz = hi.z - hj.z;
    return (qx * qx + qy * qy) * wxy_h + qz * qz * wz_h > out_lim;
}

// Screen value f of one pair-time that is not certainly outside (hi and lo
// parts of both positions): ||f_c|| = |Delta| max(0, 1/s - 1) in float32.
// Delta = (hi_i - hi_j) + (lo_i - lo_j): each rounding is relative to its own
// result, so Delta keeps a relative error of about 2 u per axis however
// close the agents are (the float pairs carry the positions to ~1e-13 C);
// |Delta| and s are then within ~3 u and ~6 u, 1/s within ~8 u, and
// |f - ||f_c||| <= 8 u rho + 4 u f <= kEpsAbs + kEpsRel f (rho <= l_max <= 1e3
// is the spheroid radius along Delta).
constexpr float kEpsRel = 2e-6f;
__device__ __forceinline__ float screen_eps(float f, float lmax) {
    return kEpsRel * (1.f + f) + 1e-6f * lmax;
}
__device__ __forceinline__ float screen_value(const float4& hi, const float4& li, const float4& hj,
                                              const float4& lj, float wxy, float wz, float lz) {
    const float dx = __fadd_rn(__fsub_rn(hi.x, hj.x), __fsub_rn(li.x, lj.x));
    const float dy = __fadd_rn(__fsub_rn(hi.y, hj.y), __fsub_rn(li.y, lj.y));
    const float dz = __fadd_rn(__fsub_rn(hi.z, hj.z), __fsub_rn(li.z, lj.z));
    float dxy, dz2;  // s^2 and its parts as pair_math.cuh forms them (each within ~3 u)
    const float s2 = pm::spheroid_s2(dx, dy, dz, wxy, wz, 0.f, dxy, dz2);
    const float nrm2 = pm::vadd(dxy, dz2);
    if (!(nrm2 >= 4.f * FLT_MIN) || !(s2 >= FLT_MIN))  // coincident to float32 range:
        return lz;                                      // u = (0, 0, l_z), reading R-degen
    if (s2 >= 1.f) return 0.f;
    // |Delta| (1/s - 1) with |Delta| = nrm2 / sqrt(nrm2)
    return nrm2 * pm::vrsqrt(nrm2) * (pm::vrsqrt(s2) - 1.f);
}

// FP64 ||f_c||^2 of the lambda-free closed form (pair_math.cuh).
__device__ __forceinline__ double free_f2_f64(double dx, double dy, double dz, double ia2,
                                              double ib2, double lz) {
    return pm::fsq_f64(dx, dy, dz, 0.0, 0.0, 0.0, ia2, ib2, lz, 0.0, 0);
}

__device__ __forceinline__ double pos64(const FreeArgs& A, int b, int ax, int ag, int t) {
    const float* xr = A.xi + ((size_t)b * 3 + ax) * A.n * A.nv + (size_t)ag * A.nv;
    double x = 0.0;
    for (int k = 0; k < A.nv; ++k) x = fma(A.P64[(size_t)t * A.nv + k], (double)xr[k], x);
    return x;
}

// FP64 ||f_c||^2 of the candidate `code` (kind << 24 | tl << 16 | i << 8 | j).
__device__ double confirm_f2(const FreeArgs& A, int b, int t0, unsigned code) {
    const int kind = code >> 24, tl = (code >> 16) & 255, i = (code >> 8) & 255, j = code & 255;
    const int t = t0 + tl;
    double d[3];
    if (kind == 0) {
        for (int ax = 0; ax < 3; ++ax) d[ax] = pos64(A, b, ax, i, t) - pos64(A, b, ax, j, t);
        return free_f2_f64(d[0], d[1], d[2], A.ia2, A.ib2, (double)A.lz);
    }
    const float* ob = A.obst + ((size_t)b * A.n_obs + j) * 5;
    for (int ax = 0; ax < 3; ++ax) d[ax] = pos64(A, b, ax, i, t) - (double)ob[ax];
    return free_f2_f64(d[0], d[1], d[2], 1.0 / ((double)ob[3] * ob[3]),
                       1.0 / ((double)ob[4] * ob[4]), (double)ob[4]);
}

// Float-pair positions of the unit's samples (and its obstacles) into shared
// memory: x = sum_k (P_hi + P_lo)[t][k] c_k with each product split exactly
// and the sum compensated; then each agent's box over the samples (hi
// parts).  Ends with a block barrier.
__device__ void unit_positions_ff(const FreeArgs& A, int b, int t0, int tcn, const FreeSmem& S) {
    // positions of the chunk's tcn <= TS samples, [agent][sample] with stride TS
    const int n = A.n, nv = A.nv, TC = A.TS, npad = A.npad;
    const float* cb = A.xi + (size_t)b * 3 * n * nv;
    for (int e = threadIdx.x; e < 3 * n * nv; e += blockDim.x) S.Cf[e] = cb[e];
    for (int e = threadIdx.x; e < tcn * nv; e += blockDim.x) {
        S.Ph[e] = A.P32[(size_t)t0 * nv + e];
        S.Pl[e] = A.P32lo[(size_t)t0 * nv + e];
    }
    for (int e = threadIdx.x; e < A.n_obs; e += blockDim.x) {
        const float* ob = A.obst + ((size_t)b * A.n_obs + e) * 5;
        const double wxy = 1.0 / ((double)ob[3] * ob[3]), wz = 1.0 / ((double)ob[4] * ob[4]);
        float* o = S.Os + e * kObstF;
        o[0] = ob[0]; o[1] = ob[1]; o[2] = ob[2];
        o[3] = (float)wxy; o[4] = (float)(wxy - (double)o[3]);
        o[5] = (float)wz; o[6] = (float)(wz - (double)o[5]);
        o[7] = ob[4];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * n * tcn; e += blockDim.x) {
        const int row = e / tcn, tl = e - row * tcn;  // row = ax * n + ag
        const float* cf = S.Cf + (size_t)row * nv;
        const float* ph = S.Ph + (size_t)tl * nv;
        const float* pl = S.Pl + (size_t)tl * nv;
        float s = 0.f, comp = 0.f;
        for (int k = 0; k < nv; ++k) {
            const float c = cf[k];
            float p, pe, te;
            two_prod(ph[k], c, p, pe);
            two_sum(s, p, s, te);
            comp = __fadd_rn(comp, __fadd_rn(te, pe));
            comp = __fmaf_rn(pl[k], c, comp);
        }
        float h, l;
        fast_two_sum(s, comp, h, l);
        const int ax = row / n, ag = row - ax * n;
        reinterpret_cast<float*>(S.Xh + (size_t)ag * TC + tl)[ax] = h;
        reinterpret_cast<float*>(S.Xl + (size_t)ag * TC + tl)[ax] = l;
        if (ax == 0) {  // the fourth components (unused) are zero
            reinterpret_cast<float*>(S.Xh + (size_t)ag * TC + tl)[3] = 0.f;
            reinterpret_cast<float*>(S.Xl + (size_t)ag * TC + tl)[3] = 0.f;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
        const int ax = e / n, ag = e - ax * n;
        const float* x = reinterpret_cast<const float*>(S.Xh + (size_t)ag * TC) + ax;
        float lo = x[0], hi = x[0];
        for (int tl = 1; tl < tcn; ++tl) { lo = fminf(lo, x[4 * tl]); hi = fmaxf(hi, x[4 * tl]); }
        S.Bx[ax * npad + ag] = lo;
        S.Bx[(3 + ax) * npad + ag] = hi;
    }
    __syncthreads();
}

// Smallest s^2 any sample of the unit can have between agent i (box) and a
// box or point j: the per-axis gap between the two intervals.
__device__ __forceinline__ float box_s2(const float* Bx, int npad, int i, float jlo0, float jhi0,
                                        float jlo1, float jhi1, float jlo2, float jhi2, float wxy,
                                        float wz) {
    const float g0 = fmaxf(0.f, fmaxf(Bx[i] - jhi0, jlo0 - Bx[3 * npad + i]));
    const float g1 = fmaxf(0.f, fmaxf(Bx[npad + i] - jhi1, jlo1 - Bx[4 * npad + i]));
    const float g2 = fmaxf(0.f, fmaxf(Bx[2 * npad + i] - jhi2, jlo2 - Bx[5 * npad + i]));
    return (g0 * g0 + g1 * g1) * wxy + g2 * g2 * wz;
}

// Screen every pair-time (and agent-obstacle row) of the unit.  MODE 0:
// keep the thread's three largest values (v[0..2]) and the codes of the
// first two.  MODE 1: FP64 recompute of every pair-time whose screen value is
// >= thr, maximum in best.  Pairs are taken in batches: phase A tests every
// pair's boxes (a thread per pair) and lists the pairs that may come close;
// phase B screens the listed pairs sample by sample (a thread per
// pair-time).  Contains block barriers: every thread of the block calls it.
struct Top3 {
    float v[3];
    unsigned c[2];
};
template <int MODE>
__device__ void screen_unit(const FreeArgs& A, int b, int t0, int tcn, const FreeSmem& Sm,
                            float out_lim, float thr, Top3& T, double& best, int* s_len) {
    // positions [agent][sample] with stride TS (the screening chunk)
    const int n = A.n, TC = A.TS, npad = A.npad, tid = threadIdx.x, bd = blockDim.x;
    const float* Bx = Sm.Bx;
    auto consider = [&](float f, unsigned code) {
        if (MODE == 0) {
            if (f > T.v[0]) {
                T.v[2] = T.v[1]; T.v[1] = T.v[0]; T.c[1] = T.c[0];
                T.v[0] = f; T.c[0] = code;
            } else if (f > T.v[1]) {
                T.v[2] = T.v[1]; T.v[1] = f; T.c[1] = code;
            } else if (f > T.v[2]) {
                T.v[2] = f;
            }
        } else if (f >= thr) {
            const double f2 = confirm_f2(A, b, t0, code);
            if (f2 > best || !(f2 == f2)) best = (f2 == f2) ? f2 : INFINITY;
        }
    };
    const float inv_tcn = 1.f / (float)tcn;
    const int p = n * (n - 1) / 2;
    // (i, j) of this thread's first pair q = tid, then advanced by bd
    int i = 0, j = 0;
    {
        int r = tid;
        while (i < n - 1 && r >= n - 1 - i) { r -= n - 1 - i; ++i; }
        j = i + 1 + r;
    }
    for (int q0 = 0; q0 < p; q0 += kPairBatch) {
        __syncthreads();  // the previous batch's list has been read
        if (tid == 0) *s_len = 0;
        __syncthreads();
        // phase A: pairs q0 .. q0 + kPairBatch - 1, a thread per pair
        for (int qq = tid; qq < kPairBatch; qq += bd) {
            const int q = q0 + qq;
            bool act = false;
            if (q < p)
                act = box_s2(Bx, npad, i, Bx[j], Bx[3 * npad + j], Bx[npad + j],
                             Bx[4 * npad + j], Bx[2 * npad + j], Bx[5 * npad + j], A.wxy_h,
                             A.wz_h) <= out_lim;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            int base = 0;
            if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(s_len, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (act)
                Sm.list[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] =
                    (unsigned short)((i << 8) | j);
            j += bd;  // advance to pair q + bd
            while (j >= n && i < n - 1) { j = j - n + i + 2; ++i; }
        }
        __syncthreads();
        // phase B: the listed pairs, a thread per (pair, sample)
        const int L = *s_len;
        for (int e = tid; e < L * tcn; e += bd) {
            const int li = __float2int_rz(((float)e + 0.5f) * inv_tcn), tl = e - li * tcn;
            const unsigned pr = Sm.list[li];
            const int pi = pr >> 8, pj = pr & 255;
            const float4 hi = Sm.Xh[pi * TC + tl], hj = Sm.Xh[pj * TC + tl];
            if (quick_outside(hi, hj, A.wxy_h, A.wz_h, out_lim)) continue;
            const float4 li4 = Sm.Xl[pi * TC + tl], lj4 = Sm.Xl[pj * TC + tl];
            consider(screen_value(hi, li4, hj, lj4, A.wxy_h, A.wz_h, A.lz),
                     ((unsigned)tl << 16) | ((unsigned)pi << 8) | (unsigned)pj);
        }
    }
    // agent-obstacle rows (reading R-obst): a thread per (agent, obstacle, sample)
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < n * A.n_obs * tcn; e += bd) {
        const int it = e / tcn, tl = e - it * tcn, ii = it / A.n_obs, o = it - ii * A.n_obs;
        const float* ob = Sm.Os + o * kObstF;
        const float4 oc = make_float4(ob[0], ob[1], ob[2], 0.f);
        const float4 hi = Sm.Xh[ii * TC + tl];
        if (quick_outside(hi, oc, ob[3], ob[5], out_lim)) continue;
        consider(screen_value(hi, Sm.Xl[ii * TC + tl], oc, zero, ob[3], ob[5], ob[7]),
                 (1u << 24) | ((unsigned)tl << 16) | ((unsigned)ii << 8) | (unsigned)o);
    }
}

constexpr int kScreenThreads = 512;
__device__ __forceinline__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
    return r;
}

// Bounds [rt - slack, rt + slack] on the true maximum of unit u (step 1).
__device__ __forceinline__ void unit_bounds(const FreeArgs& A, int b, int u, float e_d,
                                            float& lo, float& hi) {
    const float rt = sqrtf(fmaxf(A.rpart[(size_t)b * A.n_chunks + u], 0.f));
    const float sm = A.spart[(size_t)b * A.n_chunks + u];
    const float dlo = A.lmin * sqrtf(fmaxf(sm, 0.f)) * (1.f - 1e-5f) - 1.7321f * e_d;
    float slack = INFINITY;
    if (dlo > 0.f && rt == rt)
        slack = 2.f * ((1.f + A.kappa / dlo) * 1.7321f * e_d + 5.f * kU * A.lmax + 1e-6f * rt);
    lo = rt - slack;
    hi = rt + slack;
}

// One block per instance: the quick outside test's limit (from the largest
// |coefficient|), the unit skip (step 1), and the screening chunks of the
// remaining units appended to the work list; every chunk's record starts
// empty.
__global__ void __launch_bounds__(128) k_final_plan(const __grid_constant__ FreeArgs A) {
    __shared__ float red[4];
    __shared__ float s_lb;
    const int b = A.list ? A.list[blockIdx.x] : blockIdx.x, tid = threadIdx.x;
    for (int sc = tid; sc < A.NS; sc += blockDim.x) {
        float* rec = A.fin + ((size_t)b * A.NS + sc) * kFinRecFloats;
        rec[0] = -1.f; rec[1] = __int_as_float(0); rec[2] = __int_as_float(0);
    }
    if (A.flags[b] & FLAG_NONFINITE) return;  // uniform over the block
    float cm = 0.f;  // largest |coefficient|: bounds every |position| of the instance
    for (int e = tid; e < 3 * A.n * A.nv; e += blockDim.x)
        cm = fmaxf(cm, fabsf(A.xi[(size_t)b * 3 * A.n * A.nv + e]));
    cm = block_max(cm, red);
    if (tid == 0) A.olim[b] = 1.f + 1e-5f + A.out_rel * cm;
    const float e_d = 24.2f * kU * cm;  // bound on each axis of Delta's float32 error
    float lbt = -INFINITY, lo, hi;
    for (int u = tid; u < A.n_chunks && A.skip; u += blockDim.x) {
        unit_bounds(A, b, u, e_d, lo, hi);
        lbt = fmaxf(lbt, lo);
    }
    const float lb = block_max(lbt, red);
    if (tid == 0) s_lb = lb;
    __syncthreads();
    for (int u = tid; u < A.n_chunks; u += blockDim.x) {
        hi = INFINITY;
        if (A.skip) unit_bounds(A, b, u, e_d, lo, hi);
        if (hi < s_lb) continue;  // the unit cannot hold the maximum
        const int per = A.TC / A.TS, s0 = u * per, s1 = min(A.NS, s0 + per);
        const unsigned at = atomicAdd(A.wctl, (unsigned)(s1 - s0));
        for (int sc = s0; sc < s1; ++sc) A.work[at + (sc - s0)] = b * A.NS + sc;
    }
}

// Persistent grid: each block takes screening chunks (instance b, chunk sc:
// TS samples) from the work list until it is exhausted.  Per chunk: the
// float-pair positions, the screen, and the chunk's record (its largest
// value, -1 if every pair-time is certainly outside, and the pair-times that
// can reach that value).
__global__ void __launch_bounds__(kScreenThreads) k_final_screen(const __grid_constant__ FreeArgs A) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ float red[kScreenThreads / 32];
    __shared__ int s_cnt, s_ovf, s_len, s_item;
    const int tid = threadIdx.x;
    const FreeSmem Sm(fsm, A.TS, A.npad, A.n_obs, A.nv);
    for (;;) {
        __syncthreads();  // the previous chunk's shared data are no longer read
        if (tid == 0) s_item = (int)atomicAdd(A.wctl + 1, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= (int)__ldcg(A.wctl)) break;  // uniform over the block
        const int wk = A.work[item], b = wk / A.NS, sc = wk - b * A.NS;
        float* rec = A.fin + ((size_t)b * A.NS + sc) * kFinRecFloats;
        const int t0 = sc * A.TS, tcn = min(A.TS, A.m - t0);
        const float out_lim = A.olim[b];
        if (tid == 0) { s_cnt = 0; s_ovf = 0; }
        unit_positions_ff(A, b, t0, tcn, Sm);
        Top3 T;
        T.v[0] = T.v[1] = T.v[2] = -1.f;  // -1: none (screen values are >= 0)
        T.c[0] = T.c[1] = 0u;
        double unused = 0.0;
        screen_unit<0>(A, b, t0, tcn, Sm, out_lim, 0.f, T, unused, &s_len);
        const float mb = block_max(T.v[0], red);
        if (mb >= 0.f) {
            // every pair-time whose true value can reach the chunk's largest one
            const float thr = mb - 2.f * screen_eps(mb, A.lmax);
            for (int h = 0; h < 2; ++h)
                if (T.v[h] >= 0.f && T.v[h] >= thr) {
                    const int slot = atomicAdd(&s_cnt, 1);
                    if (slot < kFinCand) {
                        rec[4 + 2 * slot] = T.v[h];
                        rec[5 + 2 * slot] = __uint_as_float(T.c[h]);
                    } else {
                        s_ovf = 1;
                    }
                }
            if (T.v[2] >= 0.f && T.v[2] >= thr) s_ovf = 1;  // this thread may hold more
        }
        __syncthreads();
        if (tid == 0) {
            rec[0] = mb;
            rec[1] = __int_as_float(min(s_cnt, kFinCand));
            rec[2] = __int_as_float(s_ovf);
        }
    }
}

// One block per instance: the FP64 values of the units' candidates within
// the window of the instance's screened maximum (a warp per unit, lanes over
// its candidates), then, for a unit whose list overflowed, a new screen with
// the instance's threshold.
__global__ void __launch_bounds__(128) k_final_confirm(const __grid_constant__ FreeArgs A) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ float red[4];
    __shared__ double dred[4];
    __shared__ int s_ovf, s_len;
    const int b = A.list ? A.list[blockIdx.x] : blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (A.flags[b] & FLAG_NONFINITE) return;
    const int NC = A.NS;
    const float* recs = A.fin + (size_t)b * NC * kFinRecFloats;
    float m = -1.f;
    for (int u = tid; u < NC; u += blockDim.x) m = fmaxf(m, recs[(size_t)u * kFinRecFloats]);
    if (tid == 0) s_ovf = 0;
    m = block_max(m, red);
    double best = 0.0;  // every pair-time certainly outside: the residual is 0
    const float thr = m - 2.f * screen_eps(m, A.lmax);
    if (m >= 0.f) {
        for (int u = warp; u < NC; u += nw) {
            const float* rec = recs + (size_t)u * kFinRecFloats;
            if (!(rec[0] >= 0.f && rec[0] >= thr)) continue;
            if (__float_as_int(rec[2]) != 0) {
                if (lane == 0) s_ovf = 1;
                continue;
            }
            const int cnt = __float_as_int(rec[1]);
            for (int k = lane; k < cnt; k += 32)
                if (rec[4 + 2 * k] >= thr) {
                    const double f2 = confirm_f2(A, b, u * A.TS, __float_as_uint(rec[5 + 2 * k]));
                    if (f2 > best || !(f2 == f2)) best = (f2 == f2) ? f2 : INFINITY;
                }
        }
    }
    __syncthreads();
    if (s_ovf) {  // rare: too many near-maximal pair-times in a chunk
        const float out_lim = A.olim[b];
        const FreeSmem Sm(fsm, A.TS, A.npad, A.n_obs, A.nv);
        for (int u = 0; u < NC; ++u) {
            const float* rec = recs + (size_t)u * kFinRecFloats;
            if (!(rec[0] >= 0.f && rec[0] >= thr) || __float_as_int(rec[2]) == 0) continue;
            const int t0 = u * A.TS, tcn = min(A.TS, A.m - t0);
            __syncthreads();
            unit_positions_ff(A, b, t0, tcn, Sm);
            Top3 T;
            screen_unit<1>(A, b, t0, tcn, Sm, out_lim, thr, T, best, &s_len);
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(kFull, best, o));
    __syncthreads();
    if (lane == 0) dred[warp] = best;
    __syncthreads();
    if (tid == 0) {
        double r = dred[0];
        for (int w = 1; w < nw; ++w) r = fmax(r, dred[w]);
        A.r64[b] = (unsigned long long)__double_as_longlong(r);
    }
}

}  // namespace

int final_free_ts(const PairGeom& g, int n) {
    // the largest divisor of TC (halving) with at most about 8192 pair-times
    // per screening chunk, so that dense chunks spread over many blocks
    const int p = n * (n - 1) / 2;
    int ts = g.TC;
    while (ts > 1 && ts % 2 == 0 && (long long)p * ts > 8192) ts /= 2;
    return ts;
}

int final_free_ns(const PairGeom& g, int n, int m) {
    const int ts = final_free_ts(g, n);
    return (m + ts - 1) / ts;
}

size_t final_free_smem(const amto_plan_s* pl) {
    return sizeof(float) * free_smem_floats(final_free_ts(pl->geo, pl->n), pl->geo.npad,
                                            pl->prm.n_obstacles, pl->nv);
}

amto_status configure_final_free(amto_plan_s* pl) {
    const size_t sm = final_free_smem(pl);
    AMTO_CUDA_TRY(raise_smem_cap((const void*)k_final_screen, sm));
    AMTO_CUDA_TRY(raise_smem_cap((const void*)k_final_confirm, sm));
    int per_sm = 0;
    AMTO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_final_screen,
                                                                kScreenThreads, sm));
    pl->fin_grid = (per_sm < 1 ? 1 : per_sm) * pl->num_sms;
    return AMTO_OK;
}

amto_status launch_final_free(amto_plan_s* pl, int batch, cudaStream_t s, const int* list,
                              int nlist) {
    const PairGeom& g = pl->geo;
    FreeArgs a{};
    a.list = list;
    a.n = pl->n; a.m = pl->m; a.nv = pl->nv; a.n_chunks = g.n_chunks; a.TC = g.TC;
    a.npad = g.npad;
    a.TS = final_free_ts(g, pl->n);
    a.NS = final_free_ns(g, pl->n, pl->m);
    a.work = pl->fin_work; a.wctl = pl->fin_ctl; a.olim = pl->fin_olim;
    // units may be skipped when the last pair pass left its unit bounds (the
    // graph loop's pair kernel; not the block solver) and there are no
    // obstacles (their spheroids are not in the Lipschitz bound)
    a.skip = (!pl->block && pl->spart && pl->prm.n_obstacles == 0) ? 1 : 0;
    const double la = pl->prm.a, lb = pl->prm.b;
    const double wxy = 1.0 / (la * la), wz = 1.0 / (lb * lb);
    a.ia2 = wxy; a.ib2 = wz;
    a.wxy_h = (float)wxy; a.wxy_l = (float)(wxy - (double)a.wxy_h);
    a.wz_h = (float)wz; a.wz_l = (float)(wz - (double)a.wz_h);
    a.lz = (float)lb;
    a.out_rel = (float)(4.0 * std::ldexp(1.0, -23) / std::min(la, lb) * 2.0 * 1.0001);
    a.lmin = (float)std::min(la, lb);
    a.lmax = (float)std::max(la, lb);
    a.kappa = (float)(std::pow(std::max(la, lb), 3) * std::fabs(wxy - wz) * 0.5 * 1.0001);
    a.xi = pl->xi; a.P32 = pl->P32; a.P32lo = pl->P32lo; a.P64 = pl->P64;
    a.flags = pl->flags; a.rpart = pl->rpart; a.spart = pl->spart; a.fin = pl->fin;
    a.r64 = pl->r64;
    a.n_obs = pl->prm.n_obstacles; a.obst = pl->obst;
    const int nb_ = list ? nlist : batch;
    const size_t sm = final_free_smem(pl);
    AMTO_CUDA_TRY(cudaMemsetAsync(pl->fin_ctl, 0, sizeof(unsigned) * 2, s));  // empty work list
    k_final_plan<<<nb_, 128, 0, s>>>(a);
    AMTO_CUDA_TRY(cudaGetLastError());
    const int grid = std::max(1, std::min(pl->fin_grid, nb_ * a.NS));
    k_final_screen<<<grid, kScreenThreads, sm, s>>>(a);
    AMTO_CUDA_TRY(cudaGetLastError());
    k_final_confirm<<<nb_, 128, sm, s>>>(a);
    AMTO_CUDA_TRY(cudaGetLastError());
    return AMTO_OK;
}

}  // namespace amto
