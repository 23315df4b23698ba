// One-block-per-instance solver: the whole loop of Algorithm 1 for one
// instance runs inside one thread block, with no launch and no grid-wide
// synchronisation between iterations.
//
// Per iteration the block forms the right-hand side [rho A_fc^T(b - A_fc xi)
// - Q xi; b_eq - A_eq xi] from its own shared-memory accumulators, applies
// the cached K^-1_top (Eq. kkt_step_x, increment form; the inverse is read
// from L2, shared by all blocks of the plan), then runs the pair step (Eq.
// sphere_project, step_d, lag_update) over all pairs and samples in chunks of
// time blocks: positions in shared memory, one thread per multiplier slot
// (the multipliers keep the batched solver's layout, so the final FP64
// residual, state read-back and warm starts are shared), the contributions
// of each pair staged in shared memory and summed per agent in partner order,
// projected through P^T into the accumulators, and the stopping rule of
// Algorithm 1 decided by the block.  The arithmetic of a pair step is the
// batched kernel's (same formulas and roundings); only the summation order
// of the per-agent sums differs.
//
// Latency-bound forms (a few instances, small n: configs 1-2 and the serving
// of single requests) run at the rate of one block instead of three launches
// per iteration; uneven batches run every instance's loop in one launch.
#include <cfloat>

#include "amto_internal.cuh"
#include "pair_math.cuh"
#include "schedule.cuh"
#include "structured.cuh"

namespace amto {
namespace {

constexpr int kBT = 512;  // threads per block
constexpr unsigned kAll = 0xffffffffu;
constexpr size_t kBlockSmemBudget = 220 * 1024;  // one 512-thread block per SM

// Shared-memory plan of one instance.
struct BlockGeo {
    int nTB;        // time blocks per chunk
    size_t bytes;   // dynamic shared memory
};

__host__ __device__ inline size_t block_fixed_floats(int n, int nv, int nb, int TB, int S) {
    const int nvn = n * nv, kdim = n * (nv + nb);
    return (size_t)2 * 3 * nvn + 3 * (size_t)kdim + (size_t)n * n * TB + (size_t)S * 64 + 64;
}
__host__ __device__ inline size_t block_tb_floats(int n, int nv, int npad, int TB, int S) {
    return (size_t)TB * nv + 3 * (size_t)TB * npad + 3 * (size_t)TB * n + 3 * (size_t)S * 64;
}

struct BlockGroup {
    int n, m, nv, nb, kdim, G, nbk, npad, S, nTB, NCb, literal;
    float ia2, ib2, bz;
    RhoSched sch;        // penalty per stage; iteration k uses stage rho_stage_of(k)
    size_t ks_top, ks_ag;  // elements between the stages of Kt and Kag
    long long lam_floats;
    const float* P;      // [m][nv] float32 basis
    const float* Q;      // [nv][nv]
    const float* Am;     // [nb][nv]
    const float* Kt;     // [stages][n nv][kdim] K^-1_top
    const float* Kag;    // [stages][2][nv][nv+nb] agent-level inverse blocks (structured apply)
    int kron;            // 1: structured apply instead of the dense product
    const float* beq;    // [B][3][n nb]
    const float* gpart;  // [B][NCb][3][n nv] partials of the initial projection
    float* xi;           // [B][3][n nv]
    float* lam0;
    float* lam1;
    int* iters;
    int* flags;
    float* rmax;
    const Ctl* ctl;      // max_iters, tol
};

struct BlockArgs {
    int ng;
    int inst_start[AMTO_MAX_MIXED_GROUPS + 1];
    BlockGroup g[AMTO_MAX_MIXED_GROUPS];
};

// The batched kernel's pair arithmetic for one sample (lane orientation; the
// float instance of pair_math.cuh's pair_core, so both round alike):
// projection, d step, f_c, multiplier update, |f_c|^2 and tt = f_c +
// lambda/rho' (rho' the penalty of the next QP solve).
template <bool LIT>
__device__ __forceinline__ void pair_step1(float dx, float dy, float dz, float sgb, float ia2,
                                           float ib2, float rho, float rinv, float rnx,
                                           float& l0, float& l1,
                                           float& l2, float& t0, float& t1, float& t2,
                                           float& fsq) {
    float s2;
    pm::pair_core<float, LIT, true, true>(dx, dy, dz, sgb, ia2, ib2, rho, rinv, rnx, l0, l1, l2,
                                          t0, t1, t2, fsq, s2);
}

template <bool LIT>
__device__ void solve_instance(const BlockGroup& A, int b, float* sm) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = A.n, m = A.m, nv = A.nv, nb = A.nb, kdim = A.kdim, nvn = n * nv;
    const int G = A.G, TB = 64 / G, S = A.S, S4 = S / 4, npad = A.npad, nbk = A.nbk;
    const int nTB = A.nTB, TCB = nTB * TB, MT = (m + TB - 1) / TB;
    __shared__ float red[kBT / 32];
    __shared__ float kscr[64];
    __shared__ int s_flag;
    // shared memory plan
    float* xs = sm;                        // [3][n nv]   trajectories
    float* gs = xs + 3 * nvn;              // [3][n nv]   P^T R accumulated over the horizon
    float* rs = gs + 3 * nvn;              // [3][kdim]   right-hand side
    int* T = reinterpret_cast<int*>(rs + 3 * kdim);  // [n][n][TB] slot of pair (a, c)
    int* SL = T + n * n * TB;              // [S 64] own, partner and sample of each slot
    float* Ps = reinterpret_cast<float*>(SL + S * 64) + 64;  // [TCB][nv]
    float* X = Ps + TCB * nv;              // [3][TCB][npad] positions
    float* R = X + 3 * TCB * npad;         // [3][TCB][n]   per-agent sums
    float* Cs = R + 3 * TCB * n;           // [3][nTB S 64] pair contributions
    const int NSL = nTB * S * 64;

    if (!(A.flags[b] & FLAG_APPLY)) return;  // done or non-finite after the initial projection
    const float* xg = A.xi + (size_t)b * 3 * nvn;
    for (int i = tid; i < 3 * nvn; i += kBT) xs[i] = xg[i];
    // pair table [c][r][a] (agent fastest: conflict-free reads in the sums
    // below): chunk-relative multiplier slot of pair (a, c) at sample r of a
    // time block, bit 30 set when a is the slot's own agent
    for (int e = tid; e < n * n * TB; e += kBT) {
        const int c = e / (n * TB), r = (e / n) % TB, a = e % n;
        int v = 0;
        if (a != c) {
            int tb, sg, ln, ts;
            float sig;
            const int lo = a < c ? a : c, hi = a < c ? c : a;
            pair_slot(lo, hi, r, G, nbk, tb, sg, ln, ts, sig);
            const int own = sig > 0.f ? lo : hi;
            v = ((sg >> 2) * 256 + ts * 128 + ln * 4 + (sg & 3)) | ((own == a) ? (1 << 30) : 0);
        }
        T[e] = v;
    }
    // slot table of a time block: own agent (bits 0-9), partner (10-19), sample
    // within the time block (20-26), bit 30 set for a slot holding a pair
    for (int j = tid; j < S * 64; j += kBT) {
        const int g4 = j >> 8, q = j & 255;
        const int sg = g4 * 4 + (q & 3), ln = (q & 127) >> 2, ts = q >> 7;
        const int tr = ln / G, l = ln % G;
        int I, J, st;
        decode_step(sg, nbk, G, I, J, st);
        const int own = I * G + l, partner = J * G + ((l + st) & (G - 1));
        const bool ok = own < n && partner < n && !(I == J && st == G / 2 && l >= G / 2);
        SL[j] = ok ? (own | (partner << 10) | ((2 * tr + ts) << 20) | (1 << 30)) : 0;
    }
    // accumulators of the initial projection: sum of its chunk partials in order
    const float* gp0 = A.gpart + (size_t)b * A.NCb * 3 * nvn;
    for (int i = tid; i < 3 * nvn; i += kBT) {
        float g = 0.f;
        for (int c = 0; c < A.NCb; ++c) g += __ldcg(gp0 + (size_t)c * 3 * nvn + i);
        gs[i] = g;
    }
    const float* beq = A.beq + (size_t)b * 3 * n * nb;
    float* lbase0 = A.lam0 + (size_t)b * A.lam_floats;
    float* lbase1 = A.lam1 + (size_t)b * A.lam_floats;
    int k_it = A.iters[b];
    __syncthreads();

    for (int guard = 0; guard <= A.ctl->max_iters + 1; ++guard) {
        // this pass solves QP k_it and closes it; the target it leaves feeds QP k_it + 1
        const int sc = rho_stage_of(k_it, A.sch.J, A.sch.E);
        const int sn = rho_stage_of(k_it + 1, A.sch.J, A.sch.E);
        const float rho = A.sch.rho[sc], rinv = A.sch.rinv[sc], rnx = A.sch.rinv[sn];
        const float* Kt = A.Kt + (size_t)sc * A.ks_top;
        const float* Kag = A.Kag + (size_t)sc * A.ks_ag;
        // right-hand side (increment form)
        for (int idx = tid; idx < 3 * kdim; idx += kBT) {
            const int ax = idx / kdim, row = idx % kdim;
            const float* xr = xs + ax * nvn;
            float v;
            if (row < nvn) {
                const int i = row / nv, k = row % nv;
                float q = 0.f;
                for (int j = 0; j < nv; ++j) q = fmaf(A.Q[k * nv + j], xr[i * nv + j], q);
                v = fmaf(rho, gs[ax * nvn + row], -q);
            } else {
                const int r0 = row - nvn, i = r0 / nb, rr = r0 % nb;
                float e = 0.f;
                for (int j = 0; j < nv; ++j) e = fmaf(A.Am[rr * nv + j], xr[i * nv + j], e);
                v = beq[ax * n * nb + r0] - e;
            }
            rs[idx] = v;
        }
        __syncthreads();
        if (A.kron) {  // structured: per agent 17 x 17 blocks, axis by axis
            for (int ax = 0; ax < 3; ++ax) {
                kron_apply_axis(rs + ax * kdim, n, nv, nb, Kag, xs + ax * nvn, kscr);
                __syncthreads();
            }
        }
        // xi += K^-1_top [g; e]: a warp takes eight rows at a time, each lane
        // four columns per step, so 32 loads of K^-1 are in flight per lane
        for (int r0 = warp * 8; !A.kron && r0 < nvn; r0 += (kBT / 32) * 8) {
            float acc[8][3];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) acc[rr][0] = acc[rr][1] = acc[rr][2] = 0.f;
            for (int c0 = 0; c0 < kdim; c0 += 128) {
                float kv[8][4];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = c0 + lane + 32 * j, r = r0 + rr;
                        kv[rr][j] = (r < nvn && c < kdim) ? __ldg(Kt + (size_t)r * kdim + c) : 0.f;
                    }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + lane + 32 * j;
                    if (c < kdim) {
                        const float x0 = rs[c], x1 = rs[kdim + c], x2 = rs[2 * kdim + c];
#pragma unroll
                        for (int rr = 0; rr < 8; ++rr) {
                            acc[rr][0] = fmaf(kv[rr][j], x0, acc[rr][0]);
                            acc[rr][1] = fmaf(kv[rr][j], x1, acc[rr][1]);
                            acc[rr][2] = fmaf(kv[rr][j], x2, acc[rr][2]);
                        }
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < 8; ++rr)
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    for (int o = 16; o > 0; o >>= 1)
                        acc[rr][ax] += __shfl_xor_sync(kAll, acc[rr][ax], o);
            if (lane == 0) {
#pragma unroll
                for (int rr = 0; rr < 8; ++rr)
                    if (r0 + rr < nvn) {
                        xs[r0 + rr] += acc[rr][0];
                        xs[nvn + r0 + rr] += acc[rr][1];
                        xs[2 * nvn + r0 + rr] += acc[rr][2];
                    }
            }
        }
        for (int i = tid; i < 3 * nvn; i += kBT) gs[i] = 0.f;
        __syncthreads();

        // pair step over the horizon, chunk by chunk
        const float* lin = ((k_it - 1) & 1) ? lbase1 : lbase0;
        float* lout = (k_it & 1) ? lbase1 : lbase0;
        float fmax2 = 0.f;
        for (int tb0 = 0; tb0 < MT; tb0 += nTB) {
            const int nch = min(nTB, MT - tb0), t0 = tb0 * TB, tcn = nch * TB;
            for (int i = tid; i < tcn * nv; i += kBT) {
                const int t = t0 + i / nv;
                Ps[i] = t < m ? A.P[(size_t)t * nv + i % nv] : 0.f;
            }
            __syncthreads();
            // positions: thread (ax, agent) fixed, samples strided (no division
            // in the loop)
            {
                const int cols = 3 * npad, rows = kBT / cols > 0 ? kBT / cols : 1;
                for (int w = tid; w < cols * rows; w += kBT) {
                    const int col = w % cols, row0 = w / cols;
                    const int ax = col / npad, ag = col % npad;
                    float cf[16];
                    const float* c = xs + ax * nvn + ag * nv;
#pragma unroll
                    for (int k = 0; k < 16; ++k) cf[k] = (k < nv && ag < n) ? c[k] : 0.f;
                    for (int tl = row0; tl < tcn; tl += rows) {
                        const float* pr = Ps + tl * nv;
                        float x = 0.f;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < nv) x = fmaf(pr[k], cf[k], x);
                        X[(ax * TCB + tl) * npad + ag] = x;
                    }
                }
            }
            __syncthreads();
            // one thread per multiplier slot (consecutive threads, consecutive
            // slots); a thread's next four slots have their multipliers loaded
            // together before any of them is computed
            // slot e = kk SP + j of the chunk (time block kk, slot j of the
            // block); the thread's slots advance by kBT, (kk, j) kept without
            // division
            const int SP = S * 64, nsl = nch * SP;
            int kk_n = tid / SP, j_n = tid - (tid / SP) * SP;
            for (int e0 = tid; e0 < nsl; e0 += 4 * kBT) {
                float lv[4][3];
                size_t li[4];
                int code[4], kkv[4], jv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    kkv[u] = kk_n;
                    jv[u] = j_n;
                    const int e = e0 + u * kBT, tb = tb0 + kk_n;
                    code[u] = e < nsl ? SL[j_n] : 0;
                    if (code[u] && tb * TB + ((code[u] >> 20) & 127) >= m) code[u] = 0;
                    li[u] = (size_t)(tb * S4 + (j_n >> 8)) * 768 + (j_n & 255);
                    lv[u][0] = code[u] ? lin[li[u]] : 0.f;
                    lv[u][1] = code[u] ? lin[li[u] + 256] : 0.f;
                    lv[u][2] = code[u] ? lin[li[u] + 512] : 0.f;
                    j_n += kBT;
                    while (j_n >= SP) {
                        j_n -= SP;
                        ++kk_n;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * kBT;
                    if (e >= nsl) break;
                    float t0v = 0.f, t1v = 0.f, t2v = 0.f;
                    if (code[u]) {
                        const int o = code[u] & 1023, pp = (code[u] >> 10) & 1023;
                        const int tl = kkv[u] * TB + ((code[u] >> 20) & 127);
                        const float* Xt = X + tl * npad;
                        const float dx = Xt[o] - Xt[pp];
                        const float dy = Xt[TCB * npad + o] - Xt[TCB * npad + pp];
                        const float dz = Xt[2 * TCB * npad + o] - Xt[2 * TCB * npad + pp];
                        float l0 = lv[u][0], l1 = lv[u][1], l2 = lv[u][2];
                        const float sgb = o < pp ? A.bz : -A.bz;
                        float fsq;
                        pair_step1<LIT>(dx, dy, dz, sgb, A.ia2, A.ib2, rho, rinv, rnx, l0, l1, l2,
                                        t0v, t1v, t2v, fsq);
                        lout[li[u]] = l0;
                        lout[li[u] + 256] = l1;
                        lout[li[u] + 512] = l2;
                        fmax2 = fmaxf(fmax2, fsq);
                    }
                    Cs[e] = t0v;
                    Cs[NSL + e] = t1v;
                    Cs[2 * NSL + e] = t2v;
                }
            }
            __syncthreads();
            // per agent and sample: sum over partners in order (own: -tt, partner: +tt)
            const int arows = kBT / n, a_me = tid % n, tl_me = tid / n;
            for (int tl = tl_me; tl_me < arows && tl < tcn; tl += arows) {
                const int a = a_me, t = t0 + tl;
                float r0 = 0.f, r1 = 0.f, r2 = 0.f;
                if (t < m) {
                    const int kk = tl / TB, r = tl - kk * TB, base = kk * S4 * 256;
                    const int* Ta = T + r * n + a;
                    for (int c = 0; c < n; ++c) {
                        if (c == a) continue;
                        const int v = Ta[c * TB * n];
                        const int ci = base + (v & ((1 << 30) - 1));
                        if (v >> 30) {
                            r0 -= Cs[ci];
                            r1 -= Cs[NSL + ci];
                            r2 -= Cs[2 * NSL + ci];
                        } else {
                            r0 += Cs[ci];
                            r1 += Cs[NSL + ci];
                            r2 += Cs[2 * NSL + ci];
                        }
                    }
                }
                R[(0 * TCB + tl) * n + a] = r0;
                R[(1 * TCB + tl) * n + a] = r1;
                R[(2 * TCB + tl) * n + a] = r2;
            }
            __syncthreads();
            // accumulators: P^T R over the chunk's samples, added chunk by chunk
            for (int i = tid; i < 3 * nvn; i += kBT) {
                const int ax = i / nvn, a = (i % nvn) / nv, k = i % nv;
                float g = 0.f;
                for (int tl = 0; tl < tcn; ++tl)
                    g = fmaf(Ps[tl * nv + k], R[(ax * TCB + tl) * n + a], g);
                gs[i] += g;
            }
            __syncthreads();
        }
        // stopping rule of Algorithm 1
        for (int o = 16; o > 0; o >>= 1) fmax2 = fmaxf(fmax2, __shfl_xor_sync(kAll, fmax2, o));
        if (lane == 0) red[warp] = fmax2;
        __syncthreads();
        if (tid == 0) {
            float r2 = 0.f;
            for (int w = 0; w < kBT / 32; ++w) r2 = fmaxf(r2, red[w]);
            const float rmx = sqrtf(r2);
            A.rmax[b] = rmx;
            int nf;
            if (!isfinite(rmx)) {
                nf = FLAG_DONE | FLAG_NONFINITE;
            } else if ((k_it >= 1 && rmx < A.ctl->tol) || k_it >= A.ctl->max_iters) {
                nf = FLAG_DONE;
            } else {
                nf = FLAG_APPLY;
                A.iters[b] = k_it + 1;
            }
            A.flags[b] = nf;
            s_flag = nf;
        }
        __syncthreads();
        if (!(s_flag & FLAG_APPLY)) break;
        ++k_it;
    }
    float* xo = A.xi + (size_t)b * 3 * nvn;
    for (int i = tid; i < 3 * nvn; i += kBT) xo[i] = xs[i];
}

template <bool LIT>
__global__ void __launch_bounds__(kBT) k_solve_block(const __grid_constant__ BlockArgs M) {
    extern __shared__ __align__(16) float bsm[];
    const int y = blockIdx.x;
    int g = 0;
    while (y >= M.inst_start[g + 1]) ++g;
    solve_instance<LIT>(M.g[g], y - M.inst_start[g], bsm);
}

}  // namespace

namespace {
BlockGeo block_geometry_of(const PairGeom& g, int n, int m, int nv, int nb) {
    const int TB = 64 / g.G, MT = (m + TB - 1) / TB;
    const size_t fixed = block_fixed_floats(n, nv, nb, TB, g.S);
    const size_t per = block_tb_floats(n, nv, g.npad, TB, g.S);
    BlockGeo bg{};
    size_t room = kBlockSmemBudget / 4 > fixed ? (kBlockSmemBudget / 4 - fixed) / per : 0;
    if (room < 1) room = 1;
    bg.nTB = (int)(room < (size_t)MT ? room : (size_t)MT);
    bg.bytes = 4 * (fixed + per * bg.nTB);
    return bg;
}
BlockGeo block_geometry(const amto_plan_s* pl) {
    return block_geometry_of(pl->geo, pl->n, pl->m, pl->nv, pl->nb);
}
}  // namespace

// AUTO: the block solver wins where one block's work per iteration is small
// (measured on B300: 4 agents, one instance: 8.5 vs 24 us per iteration;
// 118 x 8 agents: 16 vs 32 us); from 16 agents on, the graph loop, which
// spreads an instance over many SMs, is faster.  One wave of blocks at most.
bool loop_block(const amto_params& p) {
    if (p.loop_mode == AMTO_LOOP_BLOCK) return true;
    if (p.loop_mode == AMTO_LOOP_GRAPH) return false;
    return p.precision == AMTO_PREC_FP32 && p.apply_mode != AMTO_APPLY_FUSED &&
           p.multipliers != AMTO_MULT_AGGREGATE && p.n_obstacles == 0 && p.n_agents <= 8 &&
           p.max_batch <= 148;
}

bool mult_aggregate(const amto_params& p) {
    if (p.multipliers != AMTO_MULT_AUTO) return p.multipliers == AMTO_MULT_AGGREGATE;
    return p.proj_mode == AMTO_PROJ_NOLAMBDA && !apply_fused(p) && !loop_block(p);
}

size_t block_solver_smem(const PairGeom& g, int n, int m, int nv, int nb) {
    return block_geometry_of(g, n, m, nv, nb).bytes;
}

amto_status configure_block_solver(amto_plan_s* pl) {
    const BlockGeo bg = block_geometry(pl);
    const void* fn = pl->prm.proj_mode == AMTO_PROJ_LITERAL ? (const void*)k_solve_block<true>
                                                            : (const void*)k_solve_block<false>;
    AMTO_CUDA_TRY(raise_smem_cap(fn, bg.bytes));
    return AMTO_OK;
}

static BlockGroup block_group(const amto_plan_s* pl) {
    const PairGeom& g = pl->geo;
    BlockGroup a{};
    a.n = pl->n; a.m = pl->m; a.nv = pl->nv; a.nb = pl->nb; a.kdim = pl->kdim;
    a.G = g.G; a.nbk = g.nbk; a.npad = g.npad; a.S = g.S; a.nTB = block_geometry(pl).nTB;
    a.NCb = g.n_chunks;
    a.literal = pl->prm.proj_mode == AMTO_PROJ_LITERAL;
    a.ia2 = (float)(1.0 / (pl->prm.a * pl->prm.a));
    a.ib2 = (float)(1.0 / (pl->prm.b * pl->prm.b));
    a.bz = (float)pl->prm.b;
    a.sch = pl->sched;
    a.ks_top = pl->ks_top;
    a.ks_ag = pl->ks_ag;
    a.lam_floats = g.lam_floats;
    a.P = pl->P32; a.Q = pl->Q32; a.Am = pl->A32; a.Kt = pl->Ktop; a.beq = pl->beq;
    a.Kag = pl->Kag;
    a.kron = pl->kron ? 1 : 0;
    a.gpart = pl->gpart; a.xi = pl->xi; a.lam0 = pl->lam[0]; a.lam1 = pl->lam[1];
    a.iters = pl->iters; a.flags = pl->flags; a.rmax = pl->rmax; a.ctl = pl->ctl;
    return a;
}

amto_status launch_block_solver(amto_plan_s* const* pls, const int* batch, int ng, cudaStream_t s) {
    if (ng < 1 || ng > AMTO_MAX_MIXED_GROUPS) {
        set_error("invalid argument: 1..AMTO_MAX_MIXED_GROUPS groups");
        return AMTO_EINVAL;
    }
    BlockArgs M{};
    M.ng = ng;
    size_t sm = 0;
    const bool lit = pls[0]->prm.proj_mode == AMTO_PROJ_LITERAL;
    for (int g = 0; g < ng; ++g) {
        M.g[g] = block_group(pls[g]);
        M.inst_start[g + 1] = M.inst_start[g] + batch[g];
        const size_t b = block_geometry(pls[g]).bytes;
        sm = b > sm ? b : sm;
        if ((pls[g]->prm.proj_mode == AMTO_PROJ_LITERAL) != lit) {
            set_error("invalid argument: the groups of one block solve share the projection mode");
            return AMTO_EINVAL;
        }
    }
    const void* fn = lit ? (const void*)k_solve_block<true> : (const void*)k_solve_block<false>;
    AMTO_CUDA_TRY(raise_smem_cap(fn, sm));
    void* args[] = {&M};
    AMTO_CUDA_TRY(cudaLaunchKernel(fn, dim3(M.inst_start[ng]), dim3(kBT), args, sm, s));
    return AMTO_OK;
}

}  // namespace amto
