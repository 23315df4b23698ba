// Mixed batches: instances with different agent counts iterated as one loop.
//
// Each agent count keeps its own plan (cached inverse, geometry, resident
// state; Remarks 1-2 make the inverse depend on n only).  A mixed solve runs
// the setup and initial projection per plan, then one loop whose body is
//   k_rhs_mixed         right-hand sides of every instance of every plan,
//   k_apply_gemm_mixed  every plan's cached-inverse GEMM tiles in one grid
//                       (+ k_splitk_reduce_mixed; tensor-core plans launch
//                       their own apply),
//   k_pair_mixed        the fused pair step: the (instance, chunk) units of
//                       all plans handed out to one persistent grid, each unit
//                       with its plan's geometry,
// captured once per combination of batch sizes as a CUDA graph under a
// conditional WHILE node; the last block of k_pair_mixed sets the condition
// from the flags of all plans.  Small and large instances therefore share
// the SMs within each launch instead of running as separate, partly empty
// launches per agent count (layout AMTO_MIXED_FUSED).  Layout
// AMTO_MIXED_BRANCHES instead runs every plan's own chain (right-hand side,
// apply, pair step) as a parallel branch of the graph body, joined by one
// kernel that sets the loop condition: the chains of different agent counts
// overlap on the device, so one count's apply runs beside another's pair
// step.  Layout AMTO_MIXED_LOOPS gives every plan its own loop: one graph
// whose parallel branches are the plans' own conditional WHILE nodes, each
// over its plan's chain with its plan's handle and control block (the
// graph of a single-plan solve, side by side), joined at the end; no count
// waits for another between iterations.
#include <map>
#include <new>
#include <string>
#include <vector>

#include "amto_internal.cuh"

struct amto_mixed_s {
    std::vector<amto_plan_s*> pls;
    int layout = AMTO_MIXED_FUSED;
    std::vector<cudaStream_t> br;      // one stream per plan (branches; setup and outputs)
    std::vector<cudaEvent_t> ev;       // fork event, then one join event per plan
    int device = 0;
    int grid = 0;                  // persistent grid of the fused pair kernel
    amto::Ctl* ctl = nullptr;      // loop control (device)
    amto::Ctl* ctl_host = nullptr; // pinned copy for the traced loop
    cudaStream_t cap = nullptr;
    bool trace = false;
    std::map<std::vector<int>, amto::Graph> graphs;
};

namespace amto {
namespace {

amto_status mixed_body(amto_mixed_s* mx, const std::vector<int>& batch,
                       cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
    const int ng = (int)mx->pls.size();
    if (mx->layout == AMTO_MIXED_BRANCHES) {
        // each plan's chain on its own stream (parallel branches of the graph
        // body), joined by one kernel that sets the loop condition
        AMTO_CUDA_TRY(cudaEventRecord(mx->ev[0], s));
        for (int g = 0; g < ng; ++g) {
            cudaStream_t b = mx->br[g];
            AMTO_CUDA_TRY(cudaStreamWaitEvent(b, mx->ev[0], 0));
            amto_status st = launch_rhs(mx->pls[g], batch[g], b);
            if (st == AMTO_OK) st = launch_apply(mx->pls[g], batch[g], b);
            if (st == AMTO_OK) st = launch_pair(mx->pls[g], batch[g], 0, nullptr, 0, 0, b);
            if (st != AMTO_OK) return st;
            AMTO_CUDA_TRY(cudaEventRecord(mx->ev[1 + g], b));
            AMTO_CUDA_TRY(cudaStreamWaitEvent(s, mx->ev[1 + g], 0));
        }
        return launch_mixed_cond(mx->pls.data(), ng, mx->ctl, h, use_cond, s);
    }
    amto_status st = launch_rhs_mixed(mx->pls.data(), batch.data(), ng, s);
    if (st == AMTO_OK) st = launch_apply_mixed(mx->pls.data(), batch.data(), ng, s);
    if (st == AMTO_OK)
        st = launch_pair_mixed(mx->pls.data(), batch.data(), ng, mx->ctl, mx->grid, h, use_cond, s);
    return st;
}

amto_status build_mixed_graph(amto_mixed_s* mx, const std::vector<int>& batch, Graph& out) {
    Graph g;
    AMTO_CUDA_TRY(cudaGraphCreate(&g.graph, 0));
    auto fail = [&](amto_status st, const char* what) {
        cudaGetLastError();
        if (what) set_error(what);
        if (g.graph) cudaGraphDestroy(g.graph);
        return st;
    };
    if (mx->layout == AMTO_MIXED_LOOPS) {
        // a WHILE node per plan, no edges between them: parallel loops
        const int ng = (int)mx->pls.size();
        for (int q = 0; q < ng; ++q) {
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, g.graph, 1, cudaGraphCondAssignDefault) !=
                cudaSuccess)
                return fail(AMTO_ECUDA, "cudaGraphConditionalHandleCreate failed");
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            if (cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp) != cudaSuccess)
                return fail(AMTO_ECUDA, "cudaGraphAddNode (while) failed");
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(mx->cap, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return fail(AMTO_ECUDA, "cudaStreamBeginCaptureToGraph failed");
            amto_plan_s* pl = mx->pls[q];
            amto_status st = launch_rhs(pl, batch[q], mx->cap);
            if (st == AMTO_OK) st = launch_apply(pl, batch[q], mx->cap);
            if (st == AMTO_OK) st = launch_pair(pl, batch[q], 0, nullptr, h, 1, mx->cap);
            cudaGraph_t captured = body;
            const cudaError_t ce = cudaStreamEndCapture(mx->cap, &captured);
            if (st != AMTO_OK) return fail(st, nullptr);
            if (ce != cudaSuccess)
                return fail(AMTO_ECUDA, "stream capture of a plan's iteration failed");
        }
        if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess)
            return fail(AMTO_ECUDA, "cudaGraphInstantiate failed");
        out = g;
        return AMTO_OK;
    }
    if (cudaGraphConditionalHandleCreate(&g.handle, g.graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess)
        return fail(AMTO_ECUDA, "cudaGraphConditionalHandleCreate failed");
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = g.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp) != cudaSuccess)
        return fail(AMTO_ECUDA, "cudaGraphAddNode (while) failed");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(mx->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(AMTO_ECUDA, "cudaStreamBeginCaptureToGraph failed");
    amto_status st = mixed_body(mx, batch, g.handle, 1, mx->cap);
    cudaGraph_t captured = body;
    const cudaError_t ce = cudaStreamEndCapture(mx->cap, &captured);
    if (st != AMTO_OK) return fail(st, nullptr);
    if (ce != cudaSuccess) return fail(AMTO_ECUDA, "stream capture of the mixed iteration failed");
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess)
        return fail(AMTO_ECUDA, "cudaGraphInstantiate failed");
    out = g;
    return AMTO_OK;
}

// Host-driven loop (profilers cannot see kernels under conditional nodes).
amto_status run_mixed_traced(amto_mixed_s* mx, const std::vector<int>& batch, int max_iters,
                             cudaStream_t s) {
    if (mx->layout == AMTO_MIXED_LOOPS) {  // every plan's chain while it has work left
        const int ng = (int)mx->pls.size();
        for (int it = 0; it <= max_iters + 1; ++it) {
            for (int q = 0; q < ng; ++q)
                AMTO_CUDA_TRY(cudaMemcpyAsync(mx->pls[q]->ctl_host, mx->pls[q]->ctl, sizeof(Ctl),
                                              cudaMemcpyDeviceToHost, s));
            AMTO_CUDA_TRY(cudaStreamSynchronize(s));
            bool any = false;
            for (int q = 0; q < ng; ++q) {
                if (mx->pls[q]->ctl_host->active_last == 0) continue;
                any = true;
                amto_status st = launch_rhs(mx->pls[q], batch[q], s);
                if (st == AMTO_OK) st = launch_apply(mx->pls[q], batch[q], s);
                if (st == AMTO_OK) st = launch_pair(mx->pls[q], batch[q], 0, nullptr, 0, 0, s);
                if (st != AMTO_OK) return st;
            }
            if (!any) break;
        }
        return AMTO_OK;
    }
    for (int it = 0; it <= max_iters + 1; ++it) {
        AMTO_CUDA_TRY(cudaMemcpyAsync(mx->ctl_host, mx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        AMTO_CUDA_TRY(cudaStreamSynchronize(s));
        if (mx->ctl_host->active_last == 0) break;
        const amto_status st = mixed_body(mx, batch, 0, 0, s);
        if (st != AMTO_OK) return st;
    }
    return AMTO_OK;
}

void free_mixed(amto_mixed_s* mx) {
    for (auto& kv : mx->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    for (cudaStream_t b : mx->br) cudaStreamDestroy(b);
    for (cudaEvent_t e : mx->ev) cudaEventDestroy(e);
    if (mx->ctl) cudaFree(mx->ctl);
    if (mx->ctl_host) cudaFreeHost(mx->ctl_host);
    if (mx->cap) cudaStreamDestroy(mx->cap);
    delete mx;
}

}  // namespace
}  // namespace amto

using namespace amto;

extern "C" {

amto_status amto_mixed_create(const amto_plan* plans, int n_plans, int layout, amto_mixed* out) {
    clear_error();
    if (!out || !plans) {
        set_error("invalid argument: plans and out are required");
        return AMTO_EINVAL;
    }
    *out = nullptr;
    if (layout != AMTO_MIXED_FUSED && layout != AMTO_MIXED_BRANCHES &&
        layout != AMTO_MIXED_LOOPS) {
        set_error("invalid argument: layout must be AMTO_MIXED_FUSED, AMTO_MIXED_BRANCHES or "
                  "AMTO_MIXED_LOOPS");
        return AMTO_EINVAL;
    }
    if (n_plans < 1 || n_plans > AMTO_MAX_MIXED_GROUPS) {
        set_error("invalid argument: n_plans must be in [1, AMTO_MAX_MIXED_GROUPS]");
        return AMTO_EINVAL;
    }
    for (int g = 0; g < n_plans; ++g) {
        const amto_plan_s* a = plans[g];
        const amto_plan_s* z = plans[0];
        if (!a) {
            set_error("invalid argument: a plan is NULL");
            return AMTO_EINVAL;
        }
        if (a->device != z->device || a->m != z->m || a->N != z->N || a->prm.T != z->prm.T ||
            a->prm.a != z->prm.a || a->prm.b != z->prm.b || a->prm.rho != z->prm.rho ||
            a->prm.bc_mask != z->prm.bc_mask || a->prm.proj_mode != z->prm.proj_mode ||
            a->prm.planar != z->prm.planar) {
            set_error("invalid argument: the plans of a mixed batch must agree on device, "
                      "m_steps, poly_degree, T, a, b, rho, bc_mask, proj_mode and planar");
            return AMTO_EINVAL;
        }
        if (a->prm.n_obstacles > 0) {
            set_error("invalid argument: mixed batches take plans without obstacles");
            return AMTO_EINVAL;
        }
        bool same_sched = a->sched.J == z->sched.J && a->sched.E == z->sched.E;
        for (int j = 0; same_sched && j < a->sched.J; ++j)
            same_sched = a->sched.rho_d[j] == z->sched.rho_d[j];
        if (!same_sched) {  // one loop count drives every group's penalty stage
            set_error("invalid argument: the plans of a mixed batch must share the rho schedule");
            return AMTO_EINVAL;
        }
        for (int h = 0; h < g; ++h)
            if (plans[h] == a) {
                set_error("invalid argument: a plan appears twice");
                return AMTO_EINVAL;
            }
    }
    amto_mixed_s* mx = new (std::nothrow) amto_mixed_s();
    if (!mx) {
        set_error("host allocation failed");
        return AMTO_ENOMEM;
    }
    mx->pls.assign(plans, plans + n_plans);
    mx->layout = layout;
    mx->device = plans[0]->device;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != mx->device) cudaSetDevice(mx->device);
    amto_status st = AMTO_OK;
    if (cudaMalloc((void**)&mx->ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void**)&mx->ctl_host, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        set_error("allocation of the mixed-batch control block failed");
        st = AMTO_ENOMEM;
    }
    if (st == AMTO_OK && cudaStreamCreateWithFlags(&mx->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaStreamCreate failed");
        st = AMTO_ECUDA;
    }
    if (st == AMTO_OK) st = configure_pair_mixed(mx->pls.data(), n_plans, &mx->grid);
    for (int g = 0; g <= n_plans && st == AMTO_OK; ++g) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaEventCreate failed");
            st = AMTO_ECUDA;
            break;
        }
        mx->ev.push_back(e);
        if (g == n_plans) break;
        cudaStream_t b = nullptr;
        if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaStreamCreate failed");
            st = AMTO_ECUDA;
            break;
        }
        mx->br.push_back(b);
    }
    if (prev >= 0 && prev != mx->device) cudaSetDevice(prev);
    if (st != AMTO_OK) {
        free_mixed(mx);
        return st;
    }
    *out = mx;
    return AMTO_OK;
}

amto_status amto_mixed_solve(amto_mixed mx, const int* batch, const float* const* start,
                             const float* const* goal, int max_iters, float tol,
                             float* const* xi_out, float* const* resid_out, int* const* iters_out,
                             void* stream) {
    clear_error();
    if (!mx || !batch || !start || !goal || !xi_out) {
        set_error("invalid argument: mixed, batch, start, goal and xi_out are required");
        return AMTO_EINVAL;
    }
    if (max_iters < 0 || !(tol >= 0.f) || !std::isfinite(tol)) {
        set_error("invalid argument: max_iters >= 0 and a finite tol >= 0 are required");
        return AMTO_EINVAL;
    }
    const int ng = (int)mx->pls.size();
    std::vector<int> b(batch, batch + ng);
    for (int g = 0; g < ng; ++g) {
        if (b[g] < 1 || b[g] > mx->pls[g]->prm.max_batch || !start[g] || !goal[g] || !xi_out[g]) {
            set_error("invalid argument: every group needs 1 <= batch <= its plan's max_batch, "
                      "start, goal and xi_out");
            return AMTO_EINVAL;
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != mx->device && cudaSetDevice(mx->device) != cudaSuccess) {
        set_error("cannot select the plans' device");
        return AMTO_ECUDA;
    }
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, mx->device};
    cudaStream_t s = (cudaStream_t)stream;
    amto_status st = launch_ctl_reset(mx->ctl, max_iters, tol, s);
    if (st != AMTO_OK) return st;
    // every plan's setup and initial projection on its own stream, in parallel
    AMTO_CUDA_TRY(cudaEventRecord(mx->ev[0], s));
    for (int g = 0; g < ng && st == AMTO_OK; ++g) {
        cudaStream_t bs = mx->br[g];
        AMTO_CUDA_TRY(cudaStreamWaitEvent(bs, mx->ev[0], 0));
        st = launch_setup(mx->pls[g], b[g], start[g], goal[g], nullptr, nullptr, max_iters, tol, bs);
        if (st == AMTO_OK) st = launch_pair(mx->pls[g], b[g], 1, nullptr, 0, 0, bs);
        if (st == AMTO_OK) {
            AMTO_CUDA_TRY(cudaEventRecord(mx->ev[1 + g], bs));
            AMTO_CUDA_TRY(cudaStreamWaitEvent(s, mx->ev[1 + g], 0));
        }
    }
    if (st != AMTO_OK) return st;
    if (mx->trace) {
        st = run_mixed_traced(mx, b, max_iters, s);
    } else {
        auto it = mx->graphs.find(b);
        if (it == mx->graphs.end()) {
            Graph gr;
            st = build_mixed_graph(mx, b, gr);
            if (st != AMTO_OK) return st;
            it = mx->graphs.emplace(b, gr).first;
        }
        AMTO_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
    }
    if (st != AMTO_OK) return st;
    // every plan's FP64 final residual and outputs on its own stream, in parallel
    AMTO_CUDA_TRY(cudaEventRecord(mx->ev[0], s));
    for (int g = 0; g < ng && st == AMTO_OK; ++g) {
        cudaStream_t bs = mx->br[g];
        AMTO_CUDA_TRY(cudaStreamWaitEvent(bs, mx->ev[0], 0));
        st = launch_final(mx->pls[g], b[g], xi_out[g], resid_out ? resid_out[g] : nullptr,
                          iters_out ? iters_out[g] : nullptr, bs);
        mx->pls[g]->last_batch = b[g];
        if (st == AMTO_OK) {
            AMTO_CUDA_TRY(cudaEventRecord(mx->ev[1 + g], bs));
            AMTO_CUDA_TRY(cudaStreamWaitEvent(s, mx->ev[1 + g], 0));
        }
    }
    return st;
}

amto_status amto_mixed_set_trace(amto_mixed mx, int on) {
    clear_error();
    if (!mx) {
        set_error("invalid argument: mixed is NULL");
        return AMTO_EINVAL;
    }
    mx->trace = on != 0;
    return AMTO_OK;
}

void amto_mixed_destroy(amto_mixed mx) {
    if (!mx) return;
    const int dev = mx->device;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    free_mixed(mx);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

}  // extern "C"
