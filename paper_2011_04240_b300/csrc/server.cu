// Serving form: continuous batching of planning requests of mixed agent counts.
//
// A server keeps one plan (cached KKT inverse, Remarks 1-2) per served agent
// count and a fixed number of resident instance slots per plan, sized from a
// device-memory budget.  A worker thread drives the GPU:
//   - newly submitted requests wait in a per-count queue and are admitted
//     into free slots between iteration chunks (the other slots keep their
//     state and keep iterating): a subset setup (boundary values, initial
//     trajectories) and a subset initial projection run for the admitted
//     slots only;
//   - every chunk, each agent-count group runs C iterations of Algorithm 1
//     for all of its resident slots as one batched step (one K^-1 GEMM per
//     group and iteration), each group on its own CUDA stream so the groups'
//     work overlaps on the device;
//   - after the chunk, slots whose stopping rule fired are retired: their
//     FP64 residual and trajectories are copied to host memory and the slot
//     is freed for the next request.
// Each instance's arithmetic depends only on its own inputs and the shared
// plan (the batched apply computes every column independently, and all
// reductions have a fixed order), so a request's result is the same alone
// and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "amto_internal.cuh"

namespace amto {

// A served count's state as the admission policy sees it: slot capacity,
// resident and queued requests, fair share and largest capacity (slots), and
// device bytes per resident instance.
struct AdmitState {
    int S, active, queued, fair, cap;
    size_t per;
};

// Device bytes of one resident instance of a plan (the state amto_create
// allocates per unit of max_batch).
size_t instance_bytes(int n, int m, int degree, unsigned bc_mask, int precision, int proj_mode) {
    // the larger multiplier layout of the two automatic lane-group choices
    const PairGeom g1 = choose_geometry(n, m, 0, 0, 1, false);
    const PairGeom g2 = choose_geometry(n, m, 0, 0, 1 << 20, false);
    const PairGeom g = g1.lam_floats >= g2.lam_floats ? g1 : g2;
    const int nv = degree + 1, nb = __builtin_popcount(bc_mask);
    const size_t kdim = (size_t)n * (nv + nb), kp = (kdim + 3) / 4 * 4, nvn = (size_t)n * nv;
    size_t b = 0;
    b += 4 * 3 * nvn;                          // xi
    b += 4 * 3 * (size_t)n * nb;               // b_eq
    // multipliers: two per-pair buffers, or A_fc^T lambda where the plan
    // aggregates them (lambda-free reading; the block solver, possible for
    // float32 plans of <= 8 agents, keeps the per-pair form)
    const bool agg = proj_mode == AMTO_PROJ_NOLAMBDA && !(precision == AMTO_PREC_FP32 && n <= 8);
    b += agg ? 4 * 3 * nvn : 2 * 4 * (size_t)g.lam_floats;
    b += 4 * (size_t)g.n_chunks * 3 * nvn;     // unit partials
    b += 2 * 4 * (size_t)g.n_chunks;           // unit maxima and smallest s^2
    {   // final-residual screening records and work list (lambda-free reading)
        const size_t ns = (size_t)final_free_ns(g, n, m);
        b += ns * (4 * (size_t)kFinRecFloats + 4) + 4;
    }
    const size_t kp8 = (kdim + 7) / 8 * 8;
    b += 4 * 3 * kp;                                            // right-hand side
    if (prec_tc(precision) && !prec_bf16(precision)) b += 4 * 3 * kp;  // TF32 lo part
    if (prec_bf16(precision)) b += 2 * 2 * 3 * kp8;             // BF16 hi / lo copies
    b += 4 * 8 * 3 * nvn;                      // split-K workspace share
    b += 48;                                   // flags, counters, precision switch
    return b;
}

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Pending {
    uint64_t ticket;
    std::vector<float> start, goal;
    double t_submit;
};

struct Result {
    int status = AMTO_EPENDING;
    int iters = 0;
    float resid = 0.f;
    std::vector<float> xi;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Group {
    int n = 0, S = 0, nv = 0;
    // memory admission: bytes of one resident instance; the capacity the
    // count gets from an equal split of the budget (its fair share) and the
    // largest it may reach (which fixes the plan's shape choices)
    size_t per = 0;
    int fair = 0, cap = 0;
    amto_params prm{};       // the plan's parameters (max_batch aside), fixed at creation
    bool tuned = false;
    amto_plan plan = nullptr;
    cudaStream_t stream = nullptr;
    float *d_start = nullptr, *d_goal = nullptr, *d_xi = nullptr, *d_resid = nullptr;
    int *d_iters = nullptr, *d_list = nullptr;
    float *h_start = nullptr, *h_goal = nullptr, *h_xi = nullptr, *h_resid = nullptr;
    int *h_iters = nullptr, *h_flags = nullptr, *h_list = nullptr;
    // chunk graphs over slot prefixes [0, pre[k]) (pre ascending, last = S):
    // admission fills the lowest free slots, so at low load a chunk launches
    // over a short prefix instead of all S slots
    std::vector<int> pre;
    std::vector<cudaGraphExec_t> chunk;
    int launched = 0;                   // prefix of the chunk in flight
    cudaEvent_t done_ev = nullptr;
    std::vector<int64_t> slot_ticket;   // -1: free
    std::vector<double> slot_admit;
    std::deque<Pending> queue;
    int active = 0;
};

}  // namespace
}  // namespace amto

struct amto_server_s {
    amto_server_params prm;
    std::vector<int> sizes;
    std::vector<std::unique_ptr<amto::Group>> groups;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<int, int> group_of_n;
    std::vector<std::deque<amto::Pending>> inbox;  // per group, guarded by mu
    std::unordered_map<uint64_t, amto::Result> results;  // guarded by mu
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int device = 0;
    size_t budget = 0, used = 0;   // bytes of resident state: the budget and the slots' share
    // statistics (guarded by mu)
    long long done_count = 0, done_iters = 0, chunks = 0, resizes = 0;
    int worker_error = AMTO_OK;
    std::string worker_msg;
};

namespace amto {
namespace {

amto_params plan_params(const amto_server_params& p, int n, int slots) {
    amto_params ap{};
    ap.n_agents = n;
    ap.m_steps = p.m_steps;
    ap.poly_degree = p.poly_degree;
    ap.T = p.T;
    ap.a = p.a;
    ap.b = p.b;
    ap.rho = p.rho;
    ap.bc_mask = AMTO_BC_ALL;
    ap.proj_mode = p.proj_mode;
    ap.precision = p.precision;
    ap.max_batch = slots;
    ap.rho_stages = p.rho_stages;
    ap.rho_growth = p.rho_growth;
    ap.rho_stage_iters = p.rho_stage_iters;
    // slots are not in step: the structured apply picks each instance's stage
    if (p.rho_stages > 1) ap.apply_mode = AMTO_APPLY_KRONECKER;
    return ap;
}

// Per-slot buffers of a group at capacity S (host staging, outputs, the
// slot list) and its chunk graphs over slot prefixes [0, pre[k]) (pre
// ascending, last = S): admission fills the lowest free slots, so at low load
// a chunk launches over a short prefix instead of all S slots.  The apply's
// split over K is fixed by the plan's reference batch, so a slot's arithmetic
// is the same in every prefix and at every capacity.
struct SlotBuffers {
    float *d_start = nullptr, *d_goal = nullptr, *d_xi = nullptr, *d_resid = nullptr;
    int *d_iters = nullptr, *d_list = nullptr;
    float *h_start = nullptr, *h_goal = nullptr, *h_xi = nullptr, *h_resid = nullptr;
    int *h_iters = nullptr, *h_flags = nullptr, *h_list = nullptr;
    std::vector<int> pre;
    std::vector<cudaGraphExec_t> chunk;
};

void buffers_free(SlotBuffers& b) {
    for (cudaGraphExec_t ex : b.chunk) cudaGraphExecDestroy(ex);
    b.chunk.clear();
    void* d[] = {b.d_start, b.d_goal, b.d_xi, b.d_resid, b.d_iters, b.d_list};
    for (void* p : d)
        if (p) cudaFree(p);
    void* h[] = {b.h_start, b.h_goal, b.h_xi, b.h_resid, b.h_iters, b.h_flags, b.h_list};
    for (void* p : h)
        if (p) cudaFreeHost(p);
    b = SlotBuffers();
}

amto_status buffers_alloc(SlotBuffers& b, int n, int nv, int S) {
    const size_t in = (size_t)S * n * 3, out = (size_t)S * 3 * n * nv;
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_start, 4 * in));
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_goal, 4 * in));
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_xi, 4 * out));
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_resid, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_iters, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMalloc((void**)&b.d_list, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_start, 4 * in));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_goal, 4 * in));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_xi, 4 * out));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_resid, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_iters, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_flags, 4 * (size_t)S));
    AMTO_CUDA_TRY(cudaMallocHost((void**)&b.h_list, 4 * (size_t)S));
    return AMTO_OK;
}

amto_status buffers_graphs(SlotBuffers& b, amto_plan_s* pl, int S, int chunk_iters,
                           cudaStream_t stream) {
    for (int q = 8; q < S; q *= 2) b.pre.push_back(q);
    b.pre.push_back(S);
    for (int q : b.pre) {
        amto_status st = AMTO_OK;
        cudaGraph_t graph;
        AMTO_CUDA_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < chunk_iters && st == AMTO_OK; ++it) {
            st = launch_rhs(pl, q, stream);
            if (st == AMTO_OK) st = launch_apply(pl, q, stream);
            if (st == AMTO_OK) st = launch_pair(pl, q, 0, nullptr, 0, 0, stream);
        }
        cudaError_t ce = cudaStreamEndCapture(stream, &graph);
        if (st != AMTO_OK) return st;
        if (ce != cudaSuccess) {
            set_error("server: capture of the iteration chunk failed");
            return AMTO_ECUDA;
        }
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            set_error("server: instantiating the iteration chunk failed");
            return AMTO_ECUDA;
        }
        b.chunk.push_back(ex);
    }
    return AMTO_OK;
}

void buffers_take(Group& g, SlotBuffers& b) {
    g.d_start = b.d_start; g.d_goal = b.d_goal; g.d_xi = b.d_xi; g.d_resid = b.d_resid;
    g.d_iters = b.d_iters; g.d_list = b.d_list;
    g.h_start = b.h_start; g.h_goal = b.h_goal; g.h_xi = b.h_xi; g.h_resid = b.h_resid;
    g.h_iters = b.h_iters; g.h_flags = b.h_flags; g.h_list = b.h_list;
    g.pre = std::move(b.pre);
    g.chunk = std::move(b.chunk);
    b = SlotBuffers();
}

SlotBuffers buffers_of(Group& g) {
    SlotBuffers b;
    b.d_start = g.d_start; b.d_goal = g.d_goal; b.d_xi = g.d_xi; b.d_resid = g.d_resid;
    b.d_iters = g.d_iters; b.d_list = g.d_list;
    b.h_start = g.h_start; b.h_goal = g.h_goal; b.h_xi = g.h_xi; b.h_resid = g.h_resid;
    b.h_iters = g.h_iters; b.h_flags = g.h_flags; b.h_list = g.h_list;
    b.pre = std::move(g.pre);
    b.chunk = std::move(g.chunk);
    g.d_start = g.d_goal = g.d_xi = g.d_resid = nullptr;
    g.d_iters = g.d_list = nullptr;
    g.h_start = g.h_goal = g.h_xi = g.h_resid = nullptr;
    g.h_iters = g.h_flags = g.h_list = nullptr;
    g.pre.clear();
    g.chunk.clear();
    return b;
}

amto_status group_init(amto_server_s* sv, Group& g, int slots) {
    const amto_server_params& p = sv->prm;
    g.S = slots;
    g.nv = p.poly_degree + 1;
    amto_params ap = g.prm;
    ap.max_batch = slots;
    amto_status st = create_plan(ap, g.cap, g.tuned, nullptr, &g.plan);
    if (st != AMTO_OK) return st;
    amto_plan_s* pl = g.plan;
    AMTO_CUDA_TRY(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    AMTO_CUDA_TRY(cudaEventCreateWithFlags(&g.done_ev, cudaEventDisableTiming));
    SlotBuffers b;
    st = buffers_alloc(b, g.n, g.nv, slots);
    if (st == AMTO_OK) st = buffers_graphs(b, pl, slots, p.chunk_iters, g.stream);
    if (st != AMTO_OK) {
        buffers_free(b);
        return st;
    }
    buffers_take(g, b);
    g.slot_ticket.assign(slots, -1);
    g.slot_admit.assign(slots, 0.0);
    // every slot starts free (flagged done, skipped by all kernels); the
    // group's stopping rule lives in the plan's control block
    std::vector<int> fl(slots, FLAG_DONE);
    AMTO_CUDA_TRY(cudaMemcpy(pl->flags, fl.data(), 4 * (size_t)slots, cudaMemcpyHostToDevice));
    Ctl c{};
    c.max_iters = p.max_iters;
    c.tol = p.tol;
    c.batch = slots;
    AMTO_CUDA_TRY(cudaMemcpy(pl->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice));
    return AMTO_OK;
}

void group_free(Group& g) {
    SlotBuffers b = buffers_of(g);
    buffers_free(b);
    if (g.done_ev) cudaEventDestroy(g.done_ev);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.plan) amto_destroy(g.plan);
}

// Change a group's capacity to S between chunks (its stream idle): a new
// plan at capacity S takes over the cached inverse and the resident
// instances' state (compacted to the lowest slots), new chunk graphs are
// captured, and the old plan is freed.  Returns AMTO_OK with the group
// unchanged if the device has no room for the new state.
amto_status group_resize(amto_server_s* sv, Group& g, int S) {
    AMTO_CUDA_TRY(cudaStreamSynchronize(g.stream));
    std::vector<int> keep;
    for (int s = 0; s < g.S; ++s)
        if (g.slot_ticket[s] >= 0) keep.push_back(s);
    if ((int)keep.size() > S || S == g.S) return AMTO_OK;
    SlotBuffers b;
    amto_status st = buffers_alloc(b, g.n, g.nv, S);
    amto_plan_s* np = nullptr;
    if (st == AMTO_OK) st = plan_resize(g.plan, S, keep.data(), (int)keep.size(), g.stream, &np);
    if (st != AMTO_OK) {
        buffers_free(b);
        if (st == AMTO_ECUDA) return st;
        clear_error();  // no room: keep the current capacity
        return AMTO_OK;
    }
    st = buffers_graphs(b, np, S, sv->prm.chunk_iters, g.stream);
    if (st != AMTO_OK) {  // keep the current capacity: the constants go back
        buffers_free(b);
        plan_give_back(np, g.plan);
        clear_error();
        return AMTO_OK;
    }
    amto_destroy(g.plan);  // its per-instance state; the constants now belong to np
    g.plan = np;
    SlotBuffers ob = buffers_of(g);
    buffers_free(ob);
    buffers_take(g, b);
    std::vector<int64_t> tk(S, -1);
    std::vector<double> ad(S, 0.0);
    for (size_t i = 0; i < keep.size(); ++i) {
        tk[i] = g.slot_ticket[keep[i]];
        ad[i] = g.slot_admit[keep[i]];
    }
    g.slot_ticket = std::move(tk);
    g.slot_admit = std::move(ad);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->used = sv->used - (size_t)g.S * g.per + (size_t)S * g.per;
    g.S = S;
    sv->resizes += 1;
    return AMTO_OK;
}

int pow2_at_least(int v) {
    int q = 1;
    while (q < v) q *= 2;
    return q;
}

}  // namespace

// One step of the shared-budget policy (see rebalance) on the counts' state,
// with no device work: the capacity changes to make, in order (donors, then
// the growing count; empty when nothing changes).
std::vector<std::pair<int, int>> admission_step(const std::vector<AdmitState>& g, size_t budget,
                                                size_t used) {
    std::vector<std::pair<int, int>> out;
    int gi = -1;
    long long unmet_best = 0;
    for (int i = 0; i < (int)g.size(); ++i) {
        const long long unmet = (long long)g[i].queued - (g[i].S - g[i].active);
        if (g[i].S < g[i].cap && unmet > unmet_best) {
            unmet_best = unmet;
            gi = i;
        }
    }
    if (gi < 0) return out;
    const AdmitState& G = g[gi];
    const int target = std::min(G.cap, std::max(2 * G.S, pow2_at_least(G.active + G.queued)));
    // donors, most reclaimable bytes first (ties: lower index)
    std::vector<std::pair<size_t, int>> donors;
    size_t room = budget > used ? budget - used : 0, avail = room;
    for (int h = 0; h < (int)g.size(); ++h) {
        if (h == gi) continue;
        const AdmitState& H = g[h];
        int floor_h = H.queued == 0
                          ? std::max(std::min(8, H.fair), pow2_at_least(std::max(H.active, 1)))
                          : std::max(H.fair, H.active);
        floor_h = std::min(floor_h, H.S);
        if (H.S - floor_h >= std::max(1, H.S / 4)) {
            donors.push_back({(size_t)(H.S - floor_h) * H.per, h});
            avail += (size_t)(H.S - floor_h) * H.per;
        }
    }
    // grow by a quarter of the capacity at least, or not at all
    const int reach = (int)std::min<size_t>((size_t)target, (size_t)G.S + avail / G.per);
    if (reach < G.S + std::max(1, G.S / 4)) return out;
    const size_t need = (size_t)(reach - G.S) * G.per;
    std::stable_sort(donors.begin(), donors.end(),
                     [](const std::pair<size_t, int>& a, const std::pair<size_t, int>& b) {
                         return a.first > b.first;
                     });
    for (const auto& d : donors) {
        if (room >= need) break;
        const AdmitState& H = g[d.second];
        out.push_back({d.second, H.S - (int)(d.first / H.per)});
        room += d.first;
    }
    const int S = (int)std::min<size_t>((size_t)reach, (size_t)G.S + room / G.per);
    if (S > G.S) out.push_back({gi, S});
    return out;
}

namespace {

// Shared memory budget (between chunks, every stream idle).  The count with
// the most queued requests beyond its free slots doubles its capacity (at
// least to the next power of two above its resident and queued requests; at
// most its largest capacity), from unclaimed budget and from the other
// counts: an idle count (empty queue) gives up free slots down to
// max(min(8, its fair share), the next power of two >= its resident
// instances); a count with a queue keeps at least its fair share.  A donor
// gives up slots only where that frees a quarter of its capacity or more, and
// a count grows only by a quarter of its capacity or more.  At most one count
// grows per chunk.
amto_status rebalance(amto_server_s* sv) {
    std::vector<AdmitState> st;
    for (auto& gp : sv->groups) {
        const Group& g = *gp;
        st.push_back({g.S, g.active, (int)std::min<size_t>(g.queue.size(), 1u << 30), g.fair,
                      g.cap, g.per});
    }
    const auto steps = admission_step(st, sv->budget, sv->used);
    for (size_t k = 0; k < steps.size(); ++k) {
        Group& g = *sv->groups[steps[k].first];
        int S = steps[k].second;
        if (k + 1 == steps.size() && S > g.S) {  // the growing count: what is actually free
            const size_t room = sv->budget > sv->used ? sv->budget - sv->used : 0;
            S = (int)std::min<size_t>((size_t)S, (size_t)g.S + room / g.per);
            if (S <= g.S) break;
        }
        const amto_status r = group_resize(sv, g, S);
        if (r != AMTO_OK) return r;
    }
    return AMTO_OK;
}

// Admit queued requests into free slots of one group (worker thread).
// At most `limit` instances resident after admission.
amto_status admit(amto_server_s* sv, Group& g, int limit) {
    int cnt = 0;
    const int n = g.n;
    for (int s = 0; s < g.S && !g.queue.empty() && g.active + cnt < limit; ++s) {
        if (g.slot_ticket[s] >= 0) continue;
        Pending p = std::move(g.queue.front());
        g.queue.pop_front();
        memcpy(g.h_start + (size_t)s * n * 3, p.start.data(), 4 * (size_t)n * 3);
        memcpy(g.h_goal + (size_t)s * n * 3, p.goal.data(), 4 * (size_t)n * 3);
        g.slot_ticket[s] = (int64_t)p.ticket;
        g.slot_admit[s] = now_s();
        g.h_list[cnt++] = s;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->results[p.ticket].t_admit = g.slot_admit[s];
        }
    }
    if (cnt == 0) return AMTO_OK;
    g.active += cnt;
    const size_t row = 4 * (size_t)n * 3;
    for (int i = 0; i < cnt; ++i) {
        const int s = g.h_list[i];
        AMTO_CUDA_TRY(cudaMemcpyAsync(g.d_start + (size_t)s * n * 3, g.h_start + (size_t)s * n * 3,
                                      row, cudaMemcpyHostToDevice, g.stream));
        AMTO_CUDA_TRY(cudaMemcpyAsync(g.d_goal + (size_t)s * n * 3, g.h_goal + (size_t)s * n * 3,
                                      row, cudaMemcpyHostToDevice, g.stream));
    }
    AMTO_CUDA_TRY(cudaMemcpyAsync(g.d_list, g.h_list, 4 * (size_t)cnt, cudaMemcpyHostToDevice,
                                  g.stream));
    amto_plan_s* pl = g.plan;
    amto_status st = launch_setup(pl, g.S, g.d_start, g.d_goal, nullptr, nullptr,
                                  sv->prm.max_iters, sv->prm.tol, g.stream, g.d_list, cnt);
    if (st == AMTO_OK) st = launch_pair(pl, g.S, 1, nullptr, 0, 0, g.stream, g.d_list, cnt);
    return st;
}

// Retire finished slots of one group (worker thread, after its chunk).
amto_status retire(amto_server_s* sv, Group& g) {
    amto_plan_s* pl = g.plan;
    int cnt = 0;
    for (int s = 0; s < g.launched; ++s)
        if (g.slot_ticket[s] >= 0 && (g.h_flags[s] & FLAG_DONE)) g.h_list[cnt++] = s;
    if (cnt == 0) return AMTO_OK;
    AMTO_CUDA_TRY(cudaMemcpyAsync(g.d_list, g.h_list, 4 * (size_t)cnt, cudaMemcpyHostToDevice,
                                  g.stream));
    amto_status st = launch_final(pl, g.S, g.d_xi, g.d_resid, g.d_iters, g.stream, g.d_list, cnt);
    if (st != AMTO_OK) return st;
    const size_t xrow = (size_t)3 * g.n * g.nv;
    for (int i = 0; i < cnt; ++i) {
        const int s = g.h_list[i];
        AMTO_CUDA_TRY(cudaMemcpyAsync(g.h_xi + s * xrow, g.d_xi + s * xrow, 4 * xrow,
                                      cudaMemcpyDeviceToHost, g.stream));
    }
    AMTO_CUDA_TRY(cudaMemcpyAsync(g.h_resid, g.d_resid, 4 * (size_t)g.launched,
                                  cudaMemcpyDeviceToHost, g.stream));
    AMTO_CUDA_TRY(cudaMemcpyAsync(g.h_iters, g.d_iters, 4 * (size_t)g.launched,
                                  cudaMemcpyDeviceToHost, g.stream));
    AMTO_CUDA_TRY(cudaStreamSynchronize(g.stream));
    const double t = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int i = 0; i < cnt; ++i) {
        const int s = g.h_list[i];
        Result& r = sv->results[(uint64_t)g.slot_ticket[s]];
        r.iters = g.h_iters[s];
        r.resid = g.h_resid[s];
        r.xi.assign(g.h_xi + s * xrow, g.h_xi + (s + 1) * xrow);
        r.t_done = t;
        r.status = r.iters == -2 ? AMTO_ETIMEOUT : r.iters < 0 ? AMTO_ENONFINITE : AMTO_OK;
        sv->done_count += 1;
        sv->done_iters += r.iters > 0 ? r.iters : 0;
        g.slot_ticket[s] = -1;
    }
    g.active -= cnt;
    sv->cv.notify_all();
    return AMTO_OK;
}

void worker_main(amto_server_s* sv) {
    cudaSetDevice(sv->device);
    amto_status st = AMTO_OK;
    while (st == AMTO_OK) {
        bool any = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            auto has_work = [&] {
                if (sv->stop) return true;
                for (size_t i = 0; i < sv->groups.size(); ++i)
                    if (!sv->inbox[i].empty() || sv->groups[i]->active > 0 ||
                        !sv->groups[i]->queue.empty())
                        return true;
                return false;
            };
            sv->cv.wait_for(lk, std::chrono::milliseconds(50), has_work);
            if (sv->stop) break;
            for (size_t i = 0; i < sv->groups.size(); ++i) {
                auto& q = sv->inbox[i];
                while (!q.empty()) {
                    sv->groups[i]->queue.push_back(std::move(q.front()));
                    q.pop_front();
                }
            }
        }
        // a count waiting below its fair share stops the counts above theirs
        // from admitting beyond them, so their capacity drains back to it
        bool starved = false;
        for (auto& gp : sv->groups)
            if (gp->S < gp->fair && gp->queue.size() > (size_t)(gp->S - gp->active)) starved = true;
        // admit, then one chunk per group with resident work (groups overlap)
        for (auto& gp : sv->groups) {
            Group& g = *gp;
            const int limit = starved && g.S > g.fair ? g.fair : g.S;
            if (st == AMTO_OK) st = admit(sv, g, limit);
            if (st == AMTO_OK && g.active > 0) {
                any = true;
                int hi = 0;
                for (int s = 0; s < g.S; ++s)
                    if (g.slot_ticket[s] >= 0) hi = s + 1;
                size_t k = 0;
                while (g.pre[k] < hi) ++k;
                g.launched = g.pre[k];
                const cudaError_t ce = cudaGraphLaunch(g.chunk[k], g.stream);
                if (ce != cudaSuccess) {
                    set_error(std::string("server: chunk launch failed: ") +
                              cudaGetErrorString(ce));
                    st = AMTO_ECUDA;
                }
                cudaMemcpyAsync(g.h_flags, g.plan->flags, 4 * (size_t)g.launched,
                                cudaMemcpyDeviceToHost, g.stream);
                cudaEventRecord(g.done_ev, g.stream);
            }
        }
        if (!any) continue;
        for (auto& gp : sv->groups) {
            Group& g = *gp;
            if (st != AMTO_OK || g.active == 0) continue;
            const cudaError_t ce = cudaEventSynchronize(g.done_ev);
            if (ce != cudaSuccess) {
                set_error(std::string("server: device error during a chunk: ") +
                          cudaGetErrorString(ce));
                st = AMTO_ECUDA;
                break;
            }
            st = retire(sv, g);
        }
        if (st == AMTO_OK && sv->prm.admission == AMTO_ADMIT_SHARED) st = rebalance(sv);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->chunks += 1;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (st != AMTO_OK) {
        sv->worker_error = st;
        sv->worker_msg = amto_last_error();
        for (auto& kv : sv->results)
            if (kv.second.status == AMTO_EPENDING) kv.second.status = st;
    }
    sv->cv.notify_all();
}

}  // namespace
}  // namespace amto

using namespace amto;

extern "C" {

amto_status amto_server_create(const amto_server_params* prm, amto_server* out) {
    clear_error();
    if (!out || !prm) {
        set_error("invalid argument: params and out are required");
        return AMTO_EINVAL;
    }
    *out = nullptr;
    const amto_server_params& p = *prm;
    if (p.n_sizes < 1 || p.n_sizes > 32 || !p.sizes) {
        set_error("invalid argument: 1..32 agent counts are required");
        return AMTO_EINVAL;
    }
    if (p.chunk_iters < 1 || p.chunk_iters > 1024 || p.max_iters < 1 || !(p.tol >= 0.f)) {
        set_error("invalid argument: chunk_iters in [1, 1024], max_iters >= 1, tol >= 0");
        return AMTO_EINVAL;
    }
    if (p.max_slots < 1 || p.max_slots > 65535) {
        set_error("invalid argument: max_slots must be in [1, 65535]");
        return AMTO_EINVAL;
    }
    if (p.admission != AMTO_ADMIT_SHARED && p.admission != AMTO_ADMIT_FIXED) {
        set_error("invalid argument: admission must be AMTO_ADMIT_SHARED or AMTO_ADMIT_FIXED");
        return AMTO_EINVAL;
    }
    for (int i = 0; i < p.n_sizes; ++i) {
        for (int j = 0; j < i; ++j)
            if (p.sizes[i] == p.sizes[j]) {
                set_error("invalid argument: agent counts must be distinct");
                return AMTO_EINVAL;
            }
        if (validate_params(plan_params(p, p.sizes[i], p.max_slots)) != AMTO_OK)
            return AMTO_EINVAL;
    }
    amto_server_s* sv = new (std::nothrow) amto_server_s();
    if (!sv) {
        set_error("host allocation failed");
        return AMTO_ENOMEM;
    }
    sv->prm = p;
    sv->sizes.assign(p.sizes, p.sizes + p.n_sizes);
    cudaGetDevice(&sv->device);
    // admission by device memory: each agent count starts at an equal share
    // of the budget (its fair share, the instances that fit in it); with the
    // shared budget a count may grow to the whole budget (at most max_slots)
    size_t budget = p.memory_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = fr / 2;
    }
    sv->budget = budget;
    const size_t share = budget / p.n_sizes;
    amto_status st = AMTO_OK;
    sv->inbox.resize(p.n_sizes);
    for (int i = 0; i < p.n_sizes && st == AMTO_OK; ++i) {
        const int n = p.sizes[i];
        const size_t per = instance_bytes(n, p.m_steps, p.poly_degree, AMTO_BC_ALL, p.precision,
                                          p.proj_mode);
        const long long fair = std::min<long long>((long long)(share / per), p.max_slots);
        const long long cap = p.admission == AMTO_ADMIT_FIXED
                                  ? fair
                                  : std::min<long long>((long long)(budget / per), p.max_slots);
        if (fair < 1) {
            set_error("server: the memory budget does not fit one instance of " + std::to_string(n) +
                      " agents");
            st = AMTO_ENOMEM;
            break;
        }
        sv->groups.emplace_back(new Group());
        sv->group_of_n[n] = i;
        Group& g = *sv->groups.back();
        g.n = n;
        g.per = per;
        g.fair = (int)fair;
        g.cap = (int)cap;
        // the shape choices (and a tuned choice, where the autotuner's cache
        // has one) are those of the largest capacity, fixed for the server's life
        g.prm = plan_params(p, n, g.cap);
        amto_params t;
        if (tune_lookup(g.prm, &t) && validate_params(t) == AMTO_OK) {
            g.prm = t;
            g.tuned = true;
        }
        clear_error();
        st = validate_params(g.prm);
        if (st == AMTO_OK) st = group_init(sv, g, g.fair);
        if (st == AMTO_OK) sv->used += (size_t)g.S * per;
    }
    if (st != AMTO_OK) {
        std::string keep = amto_last_error();
        for (auto& g : sv->groups) group_free(*g);
        delete sv;
        set_error(keep);
        return st;
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return AMTO_OK;
}

amto_status amto_server_submit(amto_server sv, const amto_request* req, uint64_t* ticket) {
    clear_error();
    if (!sv || !req || !ticket || !req->start || !req->goal) {
        set_error("invalid argument: server, request (with start and goal) and ticket are required");
        return AMTO_EINVAL;
    }
    auto it = sv->group_of_n.find(req->n_agents);
    if (it == sv->group_of_n.end()) {
        set_error("invalid argument: this server does not serve " + std::to_string(req->n_agents) +
                  " agents");
        return AMTO_EINVAL;
    }
    Pending p;
    p.start.assign(req->start, req->start + (size_t)req->n_agents * 3);
    p.goal.assign(req->goal, req->goal + (size_t)req->n_agents * 3);
    p.t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->worker_error != AMTO_OK) {
        set_error("server worker stopped: " + sv->worker_msg);
        return (amto_status)sv->worker_error;
    }
    p.ticket = sv->next_ticket++;
    Result r;
    r.t_submit = p.t_submit;
    sv->results[p.ticket] = std::move(r);
    *ticket = p.ticket;
    sv->inbox[it->second].push_back(std::move(p));
    sv->cv.notify_all();
    return AMTO_OK;
}

amto_status amto_server_poll(amto_server sv, uint64_t ticket, int wait_ms, float* xi_out,
                             amto_result_info* info) {
    clear_error();
    if (!sv) {
        set_error("invalid argument: server is NULL");
        return AMTO_EINVAL;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) {
        set_error("invalid argument: unknown or already collected ticket");
        return AMTO_EINVAL;
    }
    if (it->second.status == AMTO_EPENDING && wait_ms > 0) {
        // look the ticket up again after every wake-up: a submit in between
        // may rehash the map and invalidate iterators
        sv->cv.wait_for(lk, std::chrono::milliseconds(wait_ms),
                        [&] { return sv->results.at(ticket).status != AMTO_EPENDING; });
        it = sv->results.find(ticket);
    }
    Result& r = it->second;
    if (r.status == AMTO_EPENDING) return AMTO_EPENDING;
    if (r.status != AMTO_OK && r.status != AMTO_ENONFINITE && r.status != AMTO_ETIMEOUT)
        set_error("server worker stopped: " + sv->worker_msg);
    if (info) {
        info->iters = r.iters;
        info->resid = r.resid;
        info->t_submit = r.t_submit;
        info->t_admit = r.t_admit;
        info->t_done = r.t_done;
    }
    if (xi_out && !r.xi.empty()) memcpy(xi_out, r.xi.data(), 4 * r.xi.size());
    const amto_status st = (amto_status)r.status;
    sv->results.erase(it);
    return st;
}

amto_status amto_admission_step(int n_counts, const int* slots, const int* active,
                                const int* queued, const int* fair_slots, const int* max_capacity,
                                const unsigned long long* bytes_per_instance,
                                unsigned long long budget, int* slots_out) {
    clear_error();
    if (n_counts < 1 || n_counts > 32 || !slots || !active || !queued || !fair_slots ||
        !max_capacity || !bytes_per_instance || !slots_out) {
        set_error("invalid argument: 1..32 counts and every array are required");
        return AMTO_EINVAL;
    }
    std::vector<AdmitState> st;
    size_t used = 0;
    for (int i = 0; i < n_counts; ++i) {
        if (slots[i] < 1 || active[i] < 0 || active[i] > slots[i] || queued[i] < 0 ||
            fair_slots[i] < 1 || max_capacity[i] < slots[i] || max_capacity[i] > 65535 ||
            bytes_per_instance[i] == 0) {
            set_error("invalid argument: need 0 <= active <= slots <= max_capacity <= 65535, "
                      "queued >= 0, fair_slots >= 1 and bytes_per_instance > 0");
            return AMTO_EINVAL;
        }
        st.push_back({slots[i], active[i], queued[i], fair_slots[i], max_capacity[i],
                      (size_t)bytes_per_instance[i]});
        used += (size_t)slots[i] * (size_t)bytes_per_instance[i];
    }
    for (int i = 0; i < n_counts; ++i) slots_out[i] = slots[i];
    for (const auto& r : admission_step(st, (size_t)budget, used)) slots_out[r.first] = r.second;
    return AMTO_OK;
}

amto_status amto_server_stats(amto_server sv, amto_server_stats_t* out) {
    clear_error();
    if (!sv || !out) {
        set_error("invalid argument: server and out are required");
        return AMTO_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    out->completed = sv->done_count;
    out->iterations = sv->done_iters;
    out->chunks = sv->chunks;
    out->n_groups = (int)sv->groups.size();
    for (int i = 0; i < (int)sv->groups.size() && i < 32; ++i) {
        out->sizes[i] = sv->groups[i]->n;
        out->slots[i] = sv->groups[i]->S;
        out->fair_slots[i] = sv->groups[i]->fair;
        out->max_capacity[i] = sv->groups[i]->cap;
    }
    out->resizes = sv->resizes;
    out->budget = sv->budget;
    out->budget_used = sv->used;
    return AMTO_OK;
}

void amto_server_destroy(amto_server sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    for (auto& g : sv->groups) group_free(*g);
    delete sv;
}

}  // extern "C"
