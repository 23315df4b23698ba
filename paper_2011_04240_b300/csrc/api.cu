// C ABI entry points (include/amto.h): validation, plan memory, the solve
// sequence and its CUDA graph with a device-side loop condition.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "amto_internal.cuh"

namespace amto {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

amto_status einval(const char* what) {
    set_error(std::string("invalid argument: ") + what);
    return AMTO_EINVAL;
}

template <typename T>
amto_status dalloc(amto_plan_s* pl, T** ptr, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc((void**)ptr, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed");
        return AMTO_ENOMEM;
    }
    pl->bytes += sizeof(T) * count;
    return AMTO_OK;
}

void free_plan(amto_plan_s* pl) {
    if (!pl) return;
    for (auto& kv : pl->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    pl->graphs.clear();
    void* ptrs[] = {pl->P32, pl->P64, pl->Q32, pl->A32, pl->E0, pl->Kag, pl->Kinv64, pl->Ktop,
                    pl->xi, pl->beq, pl->lam[0], pl->lam[1], pl->Lagg, pl->obst, pl->gpart, pl->rpart, pl->spart, pl->P32lo, pl->fin, pl->fin_work, pl->fin_ctl, pl->fin_olim, pl->rhs,
                    pl->rmax, pl->r64, pl->iters, pl->flags, pl->px3, pl->pbest, pl->pat, pl->uticket, pl->gemm_ws,
                    pl->Kt_hi, pl->Kt_lo, pl->rhs_lo, pl->Kb_hi, pl->Kb_lo, pl->rb_hi, pl->rb_lo,
                    pl->gemm_tk, pl->ctl, pl->l2_flush};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (pl->ctl_host) cudaFreeHost(pl->ctl_host);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    delete pl;
}

amto_status build_graph(amto_plan_s* pl, int batch, Graph& out) {
    Graph g;
    AMTO_CUDA_TRY(cudaGraphCreate(&g.graph, 0));
    auto fail = [&](amto_status st) {
        if (g.graph) cudaGraphDestroy(g.graph);
        return st;
    };
    if (cudaGraphConditionalHandleCreate(&g.handle, g.graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGraphConditionalHandleCreate failed");
        return fail(AMTO_ECUDA);
    }
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = g.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGraphAddNode (while) failed");
        return fail(AMTO_ECUDA);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(pl->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaStreamBeginCaptureToGraph failed");
        return fail(AMTO_ECUDA);
    }
    amto_status st = launch_rhs(pl, batch, pl->cap_stream);
    if (st == AMTO_OK) st = launch_apply(pl, batch, pl->cap_stream);
    if (st == AMTO_OK) st = launch_pair(pl, batch, 0, nullptr, g.handle, 1, pl->cap_stream);
    cudaGraph_t captured = body;
    cudaError_t ce = cudaStreamEndCapture(pl->cap_stream, &captured);
    if (st != AMTO_OK) return fail(st);
    if (ce != cudaSuccess) {
        set_error(std::string("stream capture of the iteration failed: ") + cudaGetErrorString(ce));
        return fail(AMTO_ECUDA);
    }
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaGraphInstantiate failed");
        return fail(AMTO_ECUDA);
    }
    out = g;
    return AMTO_OK;
}

constexpr size_t kFlushBytes = (size_t)256 << 20;  // twice the L2 cache

__global__ void k_flush_l2(float4* buf, size_t n, float v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        buf[i] = make_float4(v, v, v, v);
}

// Host-driven loop with CUDA events around every launch (amto_set_trace).
// The loop runs while the last pair pass left an instance flagged to
// iterate, at most max_iters + 1 passes (the same bound as the graph loop).
amto_status run_traced(amto_plan_s* pl, int batch, int max_iters, cudaStream_t s) {
    cudaEvent_t ev[4];
    for (auto& e : ev) AMTO_CUDA_TRY(cudaEventCreate(&e));
    amto_status st = AMTO_OK;
    for (int it = 0; it <= max_iters + 1 && st == AMTO_OK; ++it) {
        cudaMemcpyAsync(pl->ctl_host, pl->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("traced solve: stream synchronisation failed");
            st = AMTO_ECUDA;
            break;
        }
        if (pl->ctl_host->active_last == 0) break;
        if (pl->trace == 2 && pl->l2_flush) {  // every kernel of the iteration starts cold
            k_flush_l2<<<4 * pl->num_sms, 512, 0, s>>>(pl->l2_flush, kFlushBytes / 16, (float)it);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("traced solve: L2 flush launch failed");
                st = AMTO_ECUDA;
                break;
            }
        }
        cudaEventRecord(ev[0], s);
        st = launch_rhs(pl, batch, s);
        cudaEventRecord(ev[1], s);
        if (st == AMTO_OK) st = launch_apply(pl, batch, s);
        cudaEventRecord(ev[2], s);
        if (st == AMTO_OK) st = launch_pair(pl, batch, 0, nullptr, 0, 0, s);
        cudaEventRecord(ev[3], s);
        if (cudaEventSynchronize(ev[3]) != cudaSuccess) {
            set_error("traced solve: event synchronisation failed");
            st = AMTO_ECUDA;
            break;
        }
        float ms = 0.f;
        const int kinds[3] = {KSTAT_RHS, KSTAT_APPLY, KSTAT_PAIR};
        for (int k = 0; k < 3; ++k) {
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            pl->stat_ms[kinds[k]] += ms;
            pl->stat_cnt[kinds[k]] += 1;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return st;
}

}  // namespace

// Checks of amto_params shared by amto_create and the server (no CUDA call).
amto_status validate_params(const amto_params& p) {
    if (p.n_agents < 2 || p.n_agents > 256) return einval("n_agents must be in [2, 256]");
    if (p.poly_degree < 2 || p.poly_degree > 15) return einval("poly_degree must be in [2, 15]");
    if (p.m_steps < p.poly_degree + 1 || p.m_steps > 4096)
        return einval("m_steps must be in [poly_degree + 1, 4096]");
    if (!(p.T > 0) || !std::isfinite(p.T)) return einval("T must be > 0");
    if (!(p.a > 0) || !std::isfinite(p.a) || !(p.b > 0) || !std::isfinite(p.b))
        return einval("a and b must be > 0");
    if (!(p.rho > 0) || !std::isfinite(p.rho)) return einval("rho must be > 0");
    if ((p.bc_mask & ~63u) || !(p.bc_mask & AMTO_BC_POS0) || !(p.bc_mask & AMTO_BC_POST))
        return einval("bc_mask must be a subset of AMTO_BC_ALL containing POS0 and POST");
    const int nb = __builtin_popcount(p.bc_mask);
    if (nb >= p.poly_degree + 1) return einval("more boundary conditions than coefficients");
    if (p.proj_mode != AMTO_PROJ_LITERAL && p.proj_mode != AMTO_PROJ_NOLAMBDA)
        return einval("proj_mode");
    if (p.prec_window < 0 || p.prec_window > 100000 || !(p.prec_drop >= 0.0) || !(p.prec_drop < 1.0))
        return einval("prec_window must be in [0, 100000] and prec_drop in [0, 1)");
    if (p.precision < AMTO_PREC_FP32 || p.precision > AMTO_PREC_BF16_ADAPT)
        return einval("precision must be one of AMTO_PREC_*");
    if (p.max_batch < 1 || p.max_batch > 65535) return einval("max_batch must be in [1, 65535]");
    if (p.apply_mode < AMTO_APPLY_AUTO || p.apply_mode > AMTO_APPLY_KRONECKER)
        return einval("apply_mode must be one of AMTO_APPLY_*");
    if (p.apply_mode == AMTO_APPLY_FUSED && p.precision != AMTO_PREC_FP32)
        return einval("the fused apply is float32 (AMTO_PREC_FP32) only");
    if (p.rho_stages < 0 || p.rho_stages > kMaxRhoStages)
        return einval("rho_stages must be in [0, 16]");
    if (p.rho_stages > 1 && (!(p.rho_growth > 0) || !std::isfinite(p.rho_growth) ||
                             p.rho_stage_iters < 1))
        return einval("an increasing-rho schedule needs rho_growth > 0 and rho_stage_iters >= 1");
    if (p.rho_stages > 1) {
        const double last = p.rho * std::pow(p.rho_growth, p.rho_stages - 1);
        if (!(last > 0) || !std::isfinite(last) || last > 1e8)
            return einval("the last rho stage must be a finite positive value <= 1e8");
    }
    if (p.loop_mode < AMTO_LOOP_AUTO || p.loop_mode > AMTO_LOOP_BLOCK)
        return einval("loop_mode must be one of AMTO_LOOP_*");
    if (p.loop_mode == AMTO_LOOP_BLOCK && p.apply_mode != AMTO_APPLY_KRONECKER &&
        (p.precision != AMTO_PREC_FP32 || p.apply_mode == AMTO_APPLY_FUSED))
        return einval("the block solver applies K^-1 in float32 (dense or structured) only");
    if (p.n_obstacles < 0 || p.n_obstacles > 64) return einval("n_obstacles must be in [0, 64]");
    if (p.planar != 0 && p.planar != 1) return einval("planar must be 0 or 1");
    if (p.n_obstacles > 0 && (p.loop_mode == AMTO_LOOP_BLOCK || p.apply_mode == AMTO_APPLY_FUSED))
        return einval("plans with obstacles run the graph loop with the batched, tensor-core or "
                      "structured apply");
    if (p.multipliers < AMTO_MULT_AUTO || p.multipliers > AMTO_MULT_AGGREGATE)
        return einval("multipliers must be one of AMTO_MULT_*");
    if (p.multipliers == AMTO_MULT_AGGREGATE) {
        if (p.proj_mode != AMTO_PROJ_NOLAMBDA)
            return einval("aggregated multipliers need AMTO_PROJ_NOLAMBDA (the literal reading "
                          "uses lambda per pair in the d step)");
        if (apply_fused(p) || loop_block(p))
            return einval("aggregated multipliers need the graph loop and the batched or "
                          "Kronecker apply");
    }
    if (p.tile_group != 0 && p.tile_group != 8 && p.tile_group != 16 && p.tile_group != 32)
        return einval("tile_group must be 0 (automatic), 8, 16 or 32");
    if (p.tile_time_blocks < 0 || p.tile_time_blocks > 8)
        return einval("tile_time_blocks must be in [0, 8]");
    {
        const PairGeom g = choose_geometry(p.n_agents, p.m_steps, p.tile_group, p.tile_time_blocks,
                                           p.max_batch, mult_aggregate(p), p.n_obstacles);
        if (pair_smem_bytes_host(p.n_agents, p.poly_degree + 1, __builtin_popcount(p.bc_mask),
                                 g.TC, g.npad, apply_fused(p), p.n_obstacles) > 227 * 1024)
            return einval("the pair-kernel tile does not fit in shared memory; use fewer "
                          "time blocks per warp");
        if (p.loop_mode == AMTO_LOOP_BLOCK &&
            block_solver_smem(g, p.n_agents, p.m_steps, p.poly_degree + 1,
                              __builtin_popcount(p.bc_mask)) > 227 * 1024)
            return einval("this instance is too large for the block solver; use AMTO_LOOP_GRAPH");
    }
    return AMTO_OK;
}

// The solve of amto_solve / amto_solve_from_aggregate (warm-start multipliers
// per pair in lambda_init, or aggregated in agg_init, at most one of them).
amto_status solve_impl(amto_plan plan, int batch, const float* start, const float* goal,
                       const float* bc_extra, const float* xi_init, const float* lambda_init,
                       const float* agg_init, int max_iters, float tol, float* xi_out,
                       float* resid_out, int* iters_out, void* stream) {
    if (!plan) return einval("plan is NULL");
    if (batch < 1 || batch > plan->prm.max_batch) return einval("batch must be in [1, max_batch]");
    if (!start || !goal || !xi_out) return einval("start, goal and xi_out are required");
    if (max_iters < 0) return einval("max_iters must be >= 0");
    if (!(tol >= 0.f) || !std::isfinite(tol)) return einval("tol must be a finite value >= 0");
    if (plan->prm.n_obstacles > 0 && batch > plan->obst_batch)
        return einval("the obstacles of this batch's instances have not been set (amto_set_obstacles)");
    DeviceGuard g(plan->device);
    if (!g.ok) {
        set_error("cannot select the plan's device");
        return AMTO_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    amto_status st = launch_setup(plan, batch, start, goal, bc_extra, xi_init, max_iters, tol, s);
    if (st != AMTO_OK) return st;
    if (plan->agg && lambda_init) st = launch_lambda_aggregate(plan, batch, lambda_init, s);
    if (st == AMTO_OK && agg_init) st = launch_lagg_set(plan, batch, agg_init, s);
    if (st != AMTO_OK) return st;
    st = launch_pair(plan, batch, lambda_init ? 2 : 1, lambda_init, 0, 0, s);
    if (st != AMTO_OK) return st;
    if (plan->block) {
        amto_plan_s* one[1] = {plan};
        st = launch_block_solver(one, &batch, 1, s);
    } else if (plan->trace) {
        for (int k = 0; k < KSTAT_N; ++k) {
            plan->stat_ms[k] = 0.0;
            plan->stat_cnt[k] = 0;
        }
        st = run_traced(plan, batch, max_iters, s);
    } else {
        auto it = plan->graphs.find(batch);
        if (it == plan->graphs.end()) {
            Graph gr;
            st = build_graph(plan, batch, gr);
            if (st != AMTO_OK) return st;
            it = plan->graphs.emplace(batch, gr).first;
        }
        AMTO_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
    }
    if (st != AMTO_OK) return st;
    st = launch_final(plan, batch, xi_out, resid_out, iters_out, s);
    plan->last_batch = batch;
    return st;
}

// The plan's constant device arrays (basis matrices and the cached inverses
// of Remarks 1-2): what a resized plan takes over from the plan it replaces.
template <class F>
void each_const(amto_plan_s* pl, F&& f) {
    f(reinterpret_cast<void*&>(pl->P32));
    f(reinterpret_cast<void*&>(pl->P64));
    f(reinterpret_cast<void*&>(pl->Q32));
    f(reinterpret_cast<void*&>(pl->A32));
    f(reinterpret_cast<void*&>(pl->E0));
    f(reinterpret_cast<void*&>(pl->Kag));
    f(reinterpret_cast<void*&>(pl->Kinv64));
    f(reinterpret_cast<void*&>(pl->Ktop));
    f(reinterpret_cast<void*&>(pl->Kt_hi));
    f(reinterpret_cast<void*&>(pl->Kt_lo));
    f(reinterpret_cast<void*&>(pl->Kb_hi));
    f(reinterpret_cast<void*&>(pl->Kb_lo));
    f(reinterpret_cast<void*&>(pl->P32lo));
}

// A plan for the (validated) parameters p whose shape choices -- the pair
// kernel's lane group, the apply kernel and its split over K, the block loop
// -- are those of a batch of ref_batch instances (ref_batch >= p.max_batch),
// so that an instance's arithmetic depends on ref_batch and not on the
// allocated capacity.  With a donor (a plan of the same parameters and
// ref_batch), the constants are taken over from it instead of recomputed:
// the donor keeps its per-instance state and no constants afterwards.  On
// failure the donor is unchanged.
amto_status create_plan(const amto_params& p, int ref_batch, bool tuned, amto_plan_s* donor,
                        amto_plan_s** out) {
    *out = nullptr;
    amto_params pc = p;  // the parameters the shape choices see
    pc.max_batch = ref_batch;
    amto_plan_s* pl = new (std::nothrow) amto_plan_s();
    if (!pl) {
        set_error("host allocation failed");
        return AMTO_ENOMEM;
    }
    pl->prm = p;
    pl->ref_batch = ref_batch;
    pl->tuned = tuned;
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        set_error("no CUDA device");
        return AMTO_ECUDA;
    }
    pl->n = p.n_agents;
    pl->m = p.m_steps;
    pl->N = p.poly_degree;
    pl->nv = p.poly_degree + 1;
    const int nb = __builtin_popcount(p.bc_mask);
    pl->nb = nb;
    pl->kdim = pl->n * (pl->nv + pl->nb);
    pl->p = pl->n * (pl->n - 1) / 2;
    pl->geo = choose_geometry(pl->n, pl->m, p.tile_group, p.tile_time_blocks, ref_batch,
                              mult_aggregate(pc), p.n_obstacles);
    pl->fused = apply_fused(p);
    {
        RhoSched& sc = pl->sched;
        sc.J = p.rho_stages > 1 ? p.rho_stages : 1;
        sc.E = p.rho_stages > 1 ? p.rho_stage_iters : 1;
        for (int j = 0; j < kMaxRhoStages; ++j) {
            const double r = j < sc.J ? p.rho * std::pow(p.rho_stages > 1 ? p.rho_growth : 1.0, j)
                                      : p.rho;
            sc.rho_d[j] = r;
            sc.rho[j] = (float)r;
            sc.rinv[j] = (float)(1.0 / r);
        }
    }
    pl->kron = p.apply_mode == AMTO_APPLY_KRONECKER;
    pl->block = loop_block(pc);
    pl->agg = mult_aggregate(pc);
    pl->kp = (pl->kdim + 3) / 4 * 4;   // 16-byte rows for the tensor-memory-access descriptors
    pl->kp8 = (pl->kdim + 7) / 8 * 8;  // the same for 2-byte elements
    const bool tc = prec_tc(p.precision), bf = prec_bf16(p.precision);
    const int B = p.max_batch, n = pl->n, nv = pl->nv, kdim = pl->kdim;
    const size_t nvn = (size_t)n * nv;

    amto_status st = AMTO_OK;
    if (cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaStreamCreate failed");
        st = AMTO_ECUDA;
    }
#define ALLOC(ptr, count) \
    if (st == AMTO_OK) st = dalloc(pl, &(ptr), (count))
    const int J = pl->sched.J;
    pl->ks_ag = (size_t)2 * nv * (nv + nb);
    pl->ks_top = nvn * kdim;
    pl->ks_tc = nvn * pl->kp;
    pl->ks_bf = nvn * pl->kp8;
    if (donor) {  // shared until the new plan is complete, then owned by it
        amto_plan_s* d = donor;
        pl->P32 = d->P32; pl->P64 = d->P64; pl->Q32 = d->Q32; pl->A32 = d->A32; pl->E0 = d->E0;
        pl->Kag = d->Kag; pl->Kinv64 = d->Kinv64; pl->Ktop = d->Ktop;
        pl->Kt_hi = d->Kt_hi; pl->Kt_lo = d->Kt_lo; pl->Kb_hi = d->Kb_hi; pl->Kb_lo = d->Kb_lo;
        pl->P32lo = d->P32lo;
        pl->kkt_check = d->kkt_check;
    } else {
        ALLOC(pl->P32, (size_t)pl->m * nv);
        ALLOC(pl->P64, (size_t)pl->m * nv);
        ALLOC(pl->Q32, (size_t)nv * nv);
        ALLOC(pl->A32, (size_t)nb * nv);
        ALLOC(pl->E0, (size_t)nv * nb);
        ALLOC(pl->Kag, J * pl->ks_ag);
        ALLOC(pl->Kinv64, (size_t)kdim * kdim);
        ALLOC(pl->Ktop, J * pl->ks_top);
        if (tc && !bf) {
            ALLOC(pl->Kt_hi, J * pl->ks_tc);
            ALLOC(pl->Kt_lo, J * pl->ks_tc);
        }
        if (bf) {
            ALLOC(pl->Kb_hi, J * pl->ks_bf);
            ALLOC(pl->Kb_lo, J * pl->ks_bf);
        }
        ALLOC(pl->P32lo, (size_t)pl->m * nv);
        pl->bytes_const = pl->bytes;
    }
    // per-instance state
    if (tc && !bf) ALLOC(pl->rhs_lo, (size_t)B * 3 * pl->kp);
    if (bf) {
        ALLOC(pl->rb_hi, (size_t)B * 3 * pl->kp8);
        ALLOC(pl->rb_lo, (size_t)B * 3 * pl->kp8);
    }
    ALLOC(pl->xi, (size_t)B * 3 * nvn);
    ALLOC(pl->beq, (size_t)B * 3 * n * nb);
    if (p.n_obstacles > 0) ALLOC(pl->obst, (size_t)B * p.n_obstacles * 5);
    if (pl->agg) {
        ALLOC(pl->Lagg, (size_t)B * 3 * nvn);
    } else {
        ALLOC(pl->lam[0], (size_t)B * pl->geo.lam_floats);
        ALLOC(pl->lam[1], (size_t)B * pl->geo.lam_floats);
    }
    ALLOC(pl->gpart, (size_t)B * pl->geo.n_chunks * 3 * nvn);
    ALLOC(pl->rpart, (size_t)B * pl->geo.n_chunks);
    ALLOC(pl->spart, (size_t)B * pl->geo.n_chunks);
    {
        const size_t ns = (size_t)final_free_ns(pl->geo, pl->n, pl->m);
        ALLOC(pl->fin, (size_t)B * ns * kFinRecFloats);
        ALLOC(pl->fin_work, (size_t)B * ns);
    }
    ALLOC(pl->fin_ctl, (size_t)2);
    ALLOC(pl->fin_olim, (size_t)B);
    ALLOC(pl->rhs, (size_t)B * 3 * pl->kp);
    ALLOC(pl->rmax, (size_t)B);
    ALLOC(pl->r64, (size_t)B);
    ALLOC(pl->iters, (size_t)B);
    ALLOC(pl->flags, (size_t)B);
    ALLOC(pl->px3, (size_t)B);
    ALLOC(pl->pbest, (size_t)B);
    ALLOC(pl->pat, (size_t)B);
    ALLOC(pl->uticket, (size_t)B);
    ALLOC(pl->ctl, (size_t)1);
    if (st == AMTO_OK) st = configure_kernels(pl);
    size_t ws_floats = 0;
    int tiles = 0;
    if (st == AMTO_OK) gemm_workspace(pl, &ws_floats, &tiles);
    ALLOC(pl->gemm_ws, ws_floats);
    ALLOC(pl->gemm_tk, (size_t)tiles);
#undef ALLOC
    if (st == AMTO_OK && (cudaMemset(pl->gemm_tk, 0, sizeof(unsigned) * tiles) != cudaSuccess ||
                          cudaMemset(pl->fin_ctl, 0, sizeof(unsigned) * 2) != cudaSuccess ||
                          cudaMemset(pl->uticket, 0, sizeof(unsigned) * B) != cudaSuccess)) {
        set_error("cudaMemset failed");
        st = AMTO_ECUDA;
    }
    if (st == AMTO_OK && cudaMallocHost((void**)&pl->ctl_host, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocHost failed");
        st = AMTO_ENOMEM;
    }
    if (st == AMTO_OK && !donor) st = precompute(pl);
    if (st == AMTO_OK && tc) st = tc_configure(pl);
    if (st == AMTO_OK && pl->block) st = configure_block_solver(pl);
    if (st == AMTO_OK && cudaMemset(pl->flags, 0, sizeof(int) * B) != cudaSuccess) {
        set_error("cudaMemset failed");
        st = AMTO_ECUDA;
    }
    if (st == AMTO_OK && cudaDeviceSynchronize() != cudaSuccess) {
        set_error("device error during plan creation");
        st = AMTO_ECUDA;
    }
    if (st != AMTO_OK) {
        std::string keep = g_last_error;
        if (donor) each_const(pl, [](void*& ptr) { ptr = nullptr; });  // still the donor's
        free_plan(pl);
        set_error(keep);
        return st;
    }
    if (donor) {  // the constants change owner
        each_const(donor, [](void*& ptr) { ptr = nullptr; });
        pl->bytes_const = donor->bytes_const;
        pl->bytes += donor->bytes_const;
        donor->bytes -= donor->bytes_const;
        donor->bytes_const = 0;
    }
    *out = pl;
    return AMTO_OK;
}

// dst row i = src row keep[i], for i < nkeep (rows of `words` 32-bit words).
__global__ void k_gather_rows(const unsigned* __restrict__ src, unsigned* __restrict__ dst,
                              long long words, const int* __restrict__ keep, int nkeep) {
    const long long total = words * nkeep;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / words, w = e - i * words;
        dst[e] = src[(long long)keep[i] * words + w];
    }
}

void plan_give_back(amto_plan_s* pl, amto_plan_s* old) {
    std::swap(old->bytes_const, pl->bytes_const);
    old->bytes += old->bytes_const;
    pl->bytes -= old->bytes_const;
    std::vector<void**> a, b;
    each_const(old, [&](void*& ptr) { a.push_back(&ptr); });
    each_const(pl, [&](void*& ptr) { b.push_back(&ptr); });
    for (size_t k = 0; k < a.size(); ++k) {
        *a[k] = *b[k];
        *b[k] = nullptr;
    }
    DeviceGuard g(pl->device);
    cudaDeviceSynchronize();
    free_plan(pl);
}

amto_status plan_resize(amto_plan_s* old, int new_batch, const int* keep, int nkeep,
                        cudaStream_t s, amto_plan_s** out) {
    *out = nullptr;
    if (new_batch < 1 || new_batch > 65535 || nkeep < 0 || nkeep > new_batch)
        return einval("resize: 0 <= kept instances <= new capacity <= 65535");
    if (new_batch > old->ref_batch)
        return einval("resize: the new capacity exceeds the plan's reference batch");
    for (int i = 0; i < nkeep; ++i)
        if (keep[i] < 0 || keep[i] >= old->prm.max_batch || (i > 0 && keep[i] <= keep[i - 1]))
            return einval("resize: kept instances must be ascending indexes of the old plan");
    amto_params p = old->prm;
    p.max_batch = new_batch;
    amto_plan_s* pl = nullptr;
    amto_status st = create_plan(p, old->ref_batch, old->tuned, old, &pl);
    if (st != AMTO_OK) return st;  // the old plan is unchanged
    // from here the new plan owns the constants; on failure they go back
    auto fail = [&](const char* what, amto_status st) {
        cudaGetLastError();
        plan_give_back(pl, old);
        set_error(std::string("resize: ") + what);
        return st;
    };
    const int B = new_batch, nvn = pl->n * pl->nv;
    std::vector<int> fl((size_t)B, FLAG_DONE);  // every slot not kept starts finished
    Ctl c{};
    int* d_keep = nullptr;
    if (cudaMalloc((void**)&d_keep, sizeof(int) * (size_t)(nkeep > 0 ? nkeep : 1)) != cudaSuccess)
        return fail("cudaMalloc failed", AMTO_ENOMEM);
    bool ok = cudaMemcpyAsync(d_keep, keep, sizeof(int) * (size_t)nkeep, cudaMemcpyHostToDevice,
                              s) == cudaSuccess &&
              cudaMemcpyAsync(pl->flags, fl.data(), sizeof(int) * (size_t)B,
                              cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(&c, old->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    // the per-instance arrays that live from setup to the final residual
    // (the final residual's screen records and work list and the split-K
    // workspace are rebuilt by every launch that reads them); r64 is the FP64
    // residual's running maximum, zeroed by the setup
    struct Row {
        void* src;
        void* dst;
        long long words;
    };
    const long long nobs5 = (long long)pl->prm.n_obstacles * 5;
    const Row rows[] = {
        {old->xi, pl->xi, 3LL * nvn},
        {old->beq, pl->beq, 3LL * pl->n * pl->nb},
        {old->obst, pl->obst, nobs5},
        {old->lam[0], pl->lam[0], pl->agg ? 0 : (long long)pl->geo.lam_floats},
        {old->lam[1], pl->lam[1], pl->agg ? 0 : (long long)pl->geo.lam_floats},
        {old->Lagg, pl->Lagg, pl->agg ? 3LL * nvn : 0},
        {old->gpart, pl->gpart, (long long)pl->geo.n_chunks * 3 * nvn},
        {old->rpart, pl->rpart, (long long)pl->geo.n_chunks},
        {old->spart, pl->spart, (long long)pl->geo.n_chunks},
        {old->rhs, pl->rhs, 3LL * pl->kp},
        {old->rhs_lo, pl->rhs_lo, pl->rhs_lo ? 3LL * pl->kp : 0},
        {old->rb_hi, pl->rb_hi, pl->rb_hi ? 3LL * pl->kp8 / 2 : 0},
        {old->rb_lo, pl->rb_lo, pl->rb_lo ? 3LL * pl->kp8 / 2 : 0},
        {old->rmax, pl->rmax, 1}, {old->iters, pl->iters, 1}, {old->flags, pl->flags, 1},
        {old->px3, pl->px3, 1}, {old->pbest, pl->pbest, 1}, {old->pat, pl->pat, 1},
        {old->uticket, pl->uticket, 1}, {old->fin_olim, pl->fin_olim, 1},
        {old->r64, pl->r64, 2},
    };
    for (const Row& r : rows) {
        if (!ok) break;
        if (r.words == 0 || nkeep == 0 || !r.src || !r.dst) continue;
        const long long total = r.words * nkeep;
        const int grid = (int)std::min<long long>((total + 255) / 256, 4LL * pl->num_sms);
        k_gather_rows<<<grid, 256, 0, s>>>((const unsigned*)r.src, (unsigned*)r.dst, r.words,
                                           d_keep, nkeep);
        ok = cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    c.batch = B;
    ok = ok && cudaMemcpy(pl->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice) == cudaSuccess;
    cudaFree(d_keep);
    if (!ok) return fail("moving the instances' state failed", AMTO_ECUDA);
    pl->trace = old->trace;
    pl->obst_batch = 0;
    if (pl->prm.n_obstacles > 0 && nkeep > 0 && keep[nkeep - 1] < old->obst_batch)
        pl->obst_batch = nkeep;
    *out = pl;
    return AMTO_OK;
}

}  // namespace amto

using namespace amto;

extern "C" {

const char* amto_last_error(void) { return g_last_error.c_str(); }

const char* amto_version(void) { return "amto 0.1 (sm_103a)"; }

amto_status amto_create(const amto_params* prm, amto_plan* out) {
    clear_error();
    if (!out) return einval("out is NULL");
    *out = nullptr;
    if (!prm) return einval("params is NULL");
    amto_params pp = *prm;
    if (pp.planar == 1) pp.b = pp.a;  // disks: the kernels' l_z is l_xy (z unused)
    if (amto::validate_params(pp) != AMTO_OK) return AMTO_EINVAL;
    // automatic tile, apply and loop: the autotuner's cached choice for this
    // shape, where one exists and is valid for these parameters
    bool tuned = false;
    {
        amto_params t;
        if (amto::tune_lookup(pp, &t)) {
            if (amto::validate_params(t) == AMTO_OK) {
                pp = t;
                tuned = true;
            } else {
                clear_error();
            }
        }
    }
    return amto::create_plan(pp, pp.max_batch, tuned, nullptr, out);
}

void amto_destroy(amto_plan plan) {
    if (!plan) return;
    DeviceGuard g(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
}

amto_status amto_solve(amto_plan plan, int batch, const float* start, const float* goal,
                       const float* bc_extra, const float* xi_init, const float* lambda_init,
                       int max_iters, float tol, float* xi_out, float* resid_out,
                       int* iters_out, void* stream) {
    clear_error();
    return solve_impl(plan, batch, start, goal, bc_extra, xi_init, lambda_init, nullptr,
                      max_iters, tol, xi_out, resid_out, iters_out, stream);
}

amto_status amto_solve_from_aggregate(amto_plan plan, int batch, const float* start,
                                      const float* goal, const float* bc_extra,
                                      const float* xi_init, const float* agg_init,
                                      int max_iters, float tol, float* xi_out,
                                      float* resid_out, int* iters_out, void* stream) {
    clear_error();
    if (!plan) return einval("plan is NULL");
    if (!plan->agg)
        return einval("amto_solve_from_aggregate needs a plan with aggregated multipliers "
                      "(AMTO_MULT_AGGREGATE); use amto_solve's lambda_init");
    if (!agg_init) return einval("agg_init is NULL");
    return solve_impl(plan, batch, start, goal, bc_extra, xi_init, nullptr, agg_init, max_iters,
                      tol, xi_out, resid_out, iters_out, stream);
}

amto_status amto_get_aggregate(amto_plan plan, int batch, float* agg_out, void* stream) {
    clear_error();
    if (!plan || !agg_out) return einval("plan and agg_out are required");
    if (!plan->agg)
        return einval("this plan keeps lambda per pair (AMTO_MULT_PAIRS); read it with "
                      "amto_get_state");
    if (batch < 1 || batch != plan->last_batch)
        return einval("batch must equal the last solve's batch");
    DeviceGuard g(plan->device);
    return launch_lagg_get(plan, batch, agg_out, (cudaStream_t)stream);
}



amto_status amto_get_state(amto_plan plan, int batch, float* lambda_out, float* alpha_out,
                           float* beta_out, float* d_out, void* stream) {
    clear_error();
    if (!plan) return einval("plan is NULL");
    if (batch < 1 || batch != plan->last_batch)
        return einval("batch must equal the last solve's batch");
    if (lambda_out && plan->agg)
        return einval("this plan keeps the multipliers aggregated (A_fc^T lambda, "
                      "AMTO_MULT_AGGREGATE); create it with AMTO_MULT_PAIRS to read them");
    DeviceGuard g(plan->device);
    return launch_state(plan, batch, lambda_out, alpha_out, beta_out, d_out, (cudaStream_t)stream);
}

// Obstacles of a planar plan in the kernels' axes: centre (y, 0, x), both
// semi-axes the disk's radius.
__global__ void k_planar_obstacles(long long count, const float* in, float* out) {
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= count) return;
    const float* s = in + o * 5;
    float* d = out + o * 5;
    d[0] = s[1];
    d[1] = 0.f;
    d[2] = s[0];
    d[3] = s[3];
    d[4] = s[3];
}

amto_status amto_set_obstacles(amto_plan plan, int batch, const float* obstacles, void* stream) {
    clear_error();
    if (!plan) return einval("plan is NULL");
    if (plan->prm.n_obstacles == 0) return einval("the plan has no obstacles (n_obstacles = 0)");
    if (batch < 1 || batch > plan->prm.max_batch) return einval("batch must be in [1, max_batch]");
    if (!obstacles) return einval("obstacles is NULL");
    DeviceGuard g(plan->device);
    const long long count = (long long)batch * plan->prm.n_obstacles;
    if (plan->prm.planar) {
        k_planar_obstacles<<<(unsigned)((count + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
            count, obstacles, plan->obst);
        AMTO_CUDA_TRY(cudaGetLastError());
    } else {
        AMTO_CUDA_TRY(cudaMemcpyAsync(plan->obst, obstacles, sizeof(float) * 5 * (size_t)count,
                                      cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    }
    if (batch > plan->obst_batch) plan->obst_batch = batch;
    return AMTO_OK;
}

amto_status amto_get_info(amto_plan plan, amto_info* out) {
    clear_error();
    if (!plan || !out) return einval("plan and out are required");
    out->n_agents = plan->n;
    out->m_steps = plan->m;
    out->nv = plan->nv;
    out->nb = plan->nb;
    out->kkt_dim = plan->kdim;
    out->group = plan->geo.G;
    out->t_chunk = plan->geo.TC;
    out->n_chunks = plan->geo.n_chunks;
    out->lambda_floats = plan->agg ? 0 : plan->geo.lam_floats;
    out->kkt_check = plan->kkt_check;
    out->device_bytes = plan->bytes;
    out->launches_per_iteration = launches_per_iteration(plan, plan->prm.max_batch);
    // setup, initial projection, final residual (the lambda-free reading's is
    // three launches: unit bounds and pair list, screen, confirmation), outputs
    out->launches_fixed = plan->prm.proj_mode == AMTO_PROJ_LITERAL ? 4 : 6;
    out->time_blocks = plan->geo.QW;
    out->apply_mode = plan->kron ? AMTO_APPLY_KRONECKER
                    : plan->fused ? AMTO_APPLY_FUSED : AMTO_APPLY_BATCHED;
    out->loop_mode = plan->block ? AMTO_LOOP_BLOCK : AMTO_LOOP_GRAPH;
    out->multipliers = plan->agg ? AMTO_MULT_AGGREGATE : AMTO_MULT_PAIRS;
    out->n_obstacles = plan->prm.n_obstacles;
    out->planar = plan->prm.planar;
    out->tuned = plan->tuned ? 1 : 0;
    if (plan->block) {
        out->launches_per_iteration = 0;
        out->launches_fixed += 1;  // the block solver
    }
    return AMTO_OK;
}

amto_status amto_get_kkt_inverse(amto_plan plan, double* out) {
    clear_error();
    if (!plan || !out) return einval("plan and out are required");
    DeviceGuard g(plan->device);
    AMTO_CUDA_TRY(cudaMemcpy(out, plan->Kinv64, sizeof(double) * (size_t)plan->kdim * plan->kdim,
                             cudaMemcpyDeviceToHost));
    return AMTO_OK;
}

amto_status amto_get_stats(amto_plan plan, double* out_ms, int* out_count) {
    clear_error();
    if (!plan || !out_ms || !out_count) return einval("plan, out_ms and out_count are required");
    for (int k = 0; k < KSTAT_N; ++k) {
        out_ms[k] = plan->stat_ms[k];
        out_count[k] = plan->stat_cnt[k];
    }
    return AMTO_OK;
}

amto_status amto_set_trace(amto_plan plan, int on) {
    clear_error();
    if (!plan) return einval("plan is NULL");
    if (on < 0 || on > 2) return einval("trace mode must be 0, 1 or 2");
    if (on == 2 && !plan->l2_flush) {
        DeviceGuard g(plan->device);
        if (cudaMalloc((void**)&plan->l2_flush, kFlushBytes) != cudaSuccess) {
            cudaGetLastError();
            plan->l2_flush = nullptr;
            set_error("cudaMalloc of the L2 flush buffer failed");
            return AMTO_ENOMEM;
        }
    }
    plan->trace = on;
    return AMTO_OK;
}

}  // extern "C"
