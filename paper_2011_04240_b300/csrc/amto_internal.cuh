// Internal declarations of the amto library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <string>

#include "amto.h"

namespace amto {

// ---------------------------------------------------------------------------
// Error handling: a thread-local message, no exceptions across the ABI.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();

#define AMTO_CUDA_TRY(call)                                                        \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::amto::set_error(std::string(#call " failed: ") + cudaGetErrorString(_e)); \
            return AMTO_ECUDA;                                                     \
        }                                                                          \
    } while (0)

// Apply precisions that run on the tensor cores, and those with BF16 operands.
inline bool prec_tc(int p) { return p != AMTO_PREC_FP32; }
inline bool prec_bf16(int p) {
    return p == AMTO_PREC_BF16X3 || p == AMTO_PREC_BF16 || p == AMTO_PREC_BF16_ADAPT;
}
// Per-instance switch from the single product to the hi/lo correction.
inline bool prec_adapt(int p) { return p == AMTO_PREC_TF32_ADAPT || p == AMTO_PREC_BF16_ADAPT; }
// Whether the right-hand side's lo part is formed (x3 modes and the switch).
inline bool prec_lo(int p) {
    return p == AMTO_PREC_TF32X3 || p == AMTO_PREC_BF16X3 || prec_adapt(p);
}
// Stall test of the switch: defaults of its window and relative drop.
constexpr int kPrecWindow = 8;
constexpr float kPrecDrop = 0.02f;
// Per-instance state of the switch (device, [B] each): switched (0/1), the
// best r_max so far and the iteration it was reached.
struct PrecState {
    int* x3;
    float* best;
    int* at;
};

// Programmatic dependent launch: the loop's kernels are launched so that the
// next one can be scheduled while the previous one drains; each of them waits
// here for its predecessor's results before touching global memory (a no-op
// when launched without the attribute).
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}


// Approximate 1/sqrt(x) and x/y with subnormals flushed.  Every call site
// passes a normal operand (x >= FLT_MIN by construction; y a squared unit
// length), where these give the same values as rsqrtf and __fdividef; they
// skip the extra instructions that subnormal support costs in the pair loops.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float div_ftz(float x, float y) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(y));
    return r;
}
// max(a, b, c) in one instruction (a NaN operand is ignored, as by fmaxf).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// min(a, b, c) in one instruction (a NaN operand is ignored, as by fminf).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline cudaError_t launch_pdl_c(const void* fn, dim3 grid, dim3 block, size_t smem,
                                cudaStream_t s, void** args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// Final-residual screen records (lambda-free reading, final_resid.cu): per
// unit its screened maximum, candidate count, overflow flag, one unused
// float, then kFinCand (value, code) pairs.
constexpr int kFinCand = 62;
constexpr int kFinRecFloats = 4 + 2 * kFinCand;

// Flags per instance (device int).
enum : int { FLAG_DONE = 1, FLAG_APPLY = 2, FLAG_NONFINITE = 4 };

// Kernel kinds traced by amto_get_stats.
enum : int { KSTAT_PAIR = 0, KSTAT_RHS = 1, KSTAT_APPLY = 2, KSTAT_N = 3 };

// Device-side control block of a solve.
struct Ctl {
    int max_iters;
    float tol;
    int batch;
    unsigned int ticket;        // last-block detection in the pair kernel
    unsigned int loop_count;    // pair-kernel passes of this solve (loop guard)
    unsigned int active_last;   // instances still iterating after the last pass
    unsigned int error;         // nonzero: a bounded device wait ran out
    int stage;                  // rho stage of the next QP solve (the batch iterates in step)
    unsigned int unit_next;     // next unit of the pair step to hand out (0 between launches)
};

// Increasing-rho schedule (Sec. IV-A): rho_j = rho_0 g^j, j < J; QP solve k
// (k >= 1) belongs to stage min(J - 1, (k - 1) / E); k = 0 (the initial
// projection, lambda = 0) to stage 0.
constexpr int kMaxRhoStages = 16;
__host__ __device__ inline int rho_stage_of(int k, int J, int E) {
    if (k < 1 || J <= 1) return 0;  // constant rho: no division
    const int s = (k - 1) / E;
    return s < J - 1 ? s : J - 1;
}
struct RhoSched {
    int J, E;
    float rho[kMaxRhoStages];
    float rinv[kMaxRhoStages];   // float(1 / rho) computed in double
    double rho_d[kMaxRhoStages];
};

// Planar plans (disks in the x-y plane) run the spheroid kernels with the
// axes permuted: kernel axis 0 holds the plane's y, axis 1 nothing (0), axis 2
// the plane's x, and l_z = l_xy, so the kernels' degenerate direction +z is
// the plane's +x (alpha = atan2(0, 0) = 0).  planar_src: the user axis a
// kernel axis reads (-1: none); planar_dst: the kernel axis a user axis
// comes from (-1: none, returned as 0).
__host__ __device__ inline int planar_src(int kernel_axis) {
    return kernel_axis == 0 ? 1 : kernel_axis == 2 ? 0 : -1;
}
__host__ __device__ inline int planar_dst(int user_axis) {
    return user_axis == 0 ? 2 : user_axis == 1 ? 0 : -1;
}

// Geometry of the pair kernel's work decomposition (see iterate.cu).
struct PairGeom {
    int G;          // agents per lane group (8, 16 or 32)
    int TPW;        // time samples per warp pass = 32 / G
    int nbk;        // agent blocks = ceil(n / G)
    int npad;       // nbk * G
    int S;          // pair steps per time group = nbk^2 G / 2 (a multiple of 4)
    int So;         // agent-obstacle steps per time group = nbk n_obs rounded up to 4
    int warps;      // warps per block
    int QW;         // time groups per warp
    int QC;         // time groups per block = warps * QW
    int TC;         // time samples per block = QC * TPW
    int n_chunks;   // work units per instance = ceil(m / TC)
    int MQ;         // time groups per instance = n_chunks * QC
    long long lam_floats;  // multiplier floats per instance and buffer = MQ * (S + So) * 3 * 32
    int grid;       // persistent pair-kernel blocks (set when the kernels are configured)
};

// Pair-kernel geometry for n agents and m samples: lane group G and time
// blocks per warp and unit QW (0: automatic, depending on the batch size).
PairGeom choose_geometry(int n, int m, int G_req, int QW_req, int max_batch, bool agg,
                         int n_obs = 0);

struct Graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
};

}  // namespace amto

struct amto_plan_s {
    amto_params prm;
    int device = 0;
    int num_sms = 0;
    int n = 0, m = 0, N = 0, nv = 0, nb = 0, kdim = 0, p = 0;
    amto::PairGeom geo{};
    double kkt_check = 0.0;
    size_t bytes = 0;          // device bytes held by the plan
    size_t bytes_const = 0;    // of which the constants (taken over by a resized plan)
    // the batch that fixes the shape choices (the pair kernel's lane group,
    // the apply kernel and its split over K, the block loop): max_batch for
    // amto_create; a resizable plan's largest capacity, so that an instance's
    // arithmetic does not depend on the capacity allocated
    int ref_batch = 0;

    // constants (device)
    float* P32 = nullptr;      // [m][nv]
    double* P64 = nullptr;     // [m][nv]
    float* Q32 = nullptr;      // [nv][nv]  Pddot^T Pddot
    float* A32 = nullptr;      // [nb][nv]
    float* E0 = nullptr;       // [nv][nb]  top-right block of the agent-level inverse
    float* Kag = nullptr;      // [2][nv][nv+nb] top rows of K_n^-1 and K_0^-1 (agent level)
    double* Kinv64 = nullptr;  // [kdim][kdim]
    float* Ktop = nullptr;     // [n nv][kdim]
    int kp = 0;                // padded row length (multiple of 4) of the tensor-core operands
    float* Kt_hi = nullptr;    // [n nv][kp] TF32-rounded K^-1_top (tensor-core modes)
    float* Kt_lo = nullptr;    // [n nv][kp] float32 residual K^-1_top - Kt_hi
    int kp8 = 0;               // padded row length (multiple of 8) of the BF16 operands
    unsigned short* Kb_hi = nullptr;  // [n nv][kp8] BF16(K^-1_top) (BF16 modes)
    unsigned short* Kb_lo = nullptr;  // [n nv][kp8] BF16(K^-1_top - Kb_hi)
    CUtensorMap tm_a_hi[amto::kMaxRhoStages], tm_a_lo[amto::kMaxRhoStages];  // K^-1 per rho stage
    CUtensorMap tm_b_hi, tm_b_lo;  // right-hand-side operands (TMA descriptors, 64-byte aligned)
    amto::RhoSched sched;      // rho stages (J = 1: constant rho)
    size_t ks_top = 0, ks_tc = 0, ks_bf = 0, ks_ag = 0;  // per-stage strides of the inverses

    // state for max_batch instances (device)
    float* xi = nullptr;       // [B][3][n nv]
    float* beq = nullptr;      // [B][3][n nb]
    float* lam[2] = {nullptr, nullptr};  // [B][lam_floats] (PAIRS form only)
    float* Lagg = nullptr;     // [B][3][n nv] A_fc^T lambda (AGGREGATE form only)
    float* obst = nullptr;     // [B][n_obs][5] obstacle centres and semi-axes (amto_set_obstacles)
    int obst_batch = 0;        // instances whose obstacles have been set
    float* gpart = nullptr;    // [B][n_chunks][3][n nv]
    float* rpart = nullptr;    // [B][n_chunks] max ||f_c||^2 of each pair-kernel unit (float32)
    float* spart = nullptr;    // [B][n_chunks] min s^2 of each unit (lambda-free reading)
    float* P32lo = nullptr;    // [m][nv] float32(P64 - P32): P64 as a float pair (final residual)
    float* fin = nullptr;      // [B][fin_ns][kFinRecFloats] final-residual screen records
    int* fin_work = nullptr;   // [B fin_ns] final-residual screening chunks to do
    unsigned* fin_ctl = nullptr;  // [2] chunks listed / taken (cleared by each final residual)
    float* fin_olim = nullptr; // [B] the final screen's outside-test limit per instance
    int fin_grid = 0;          // persistent blocks of the final screen
    float* rhs = nullptr;      // [B][3][kp] (TF32-rounded in tensor-core modes)
    float* rhs_lo = nullptr;   // [B][3][kp] residual rhs - rhs (TF32X3 mode)
    unsigned short* rb_hi = nullptr;  // [B][3][kp8] BF16(rhs) (BF16 modes)
    unsigned short* rb_lo = nullptr;  // [B][3][kp8] BF16(rhs - rb_hi) (BF16X3 mode)
    float* rmax = nullptr;     // [B]
    unsigned long long* r64 = nullptr;  // [B] FP64 final residual^2 bits
    int* iters = nullptr;      // [B]
    int* flags = nullptr;      // [B]
    int* px3 = nullptr;        // [B] hi/lo correction switched on (AMTO_PREC_*_ADAPT)
    float* pbest = nullptr;    // [B] best r_max so far (the switch's stall test)
    int* pat = nullptr;        // [B] iteration of that best value
    unsigned* uticket = nullptr;  // [B] finished pair-kernel units per instance
    float* gemm_ws = nullptr;     // split-K partial products of the SIMT apply
    unsigned* gemm_tk = nullptr;  // per-tile tickets of the split-K reduction
    amto::Ctl* ctl = nullptr;
    amto::Ctl* ctl_host = nullptr;   // pinned mirror for host polling

    int last_batch = 0;
    bool fused = false;        // K^-1 applied per instance inside the pair kernel
    bool block = false;        // the loop runs in the one-block-per-instance solver
    bool kron = false;         // K^-1 applied in its exact agent-structured form
    bool agg = false;          // multipliers kept as A_fc^T lambda (AMTO_MULT_AGGREGATE)
    bool tuned = false;        // tile, apply and loop taken from the autotuner's cache
    cudaStream_t cap_stream = nullptr;
    std::map<int, amto::Graph> graphs;

    // tracing
    int trace = 0;               // 0 graph loop, 1 traced loop, 2 traced with L2 flushes
    float4* l2_flush = nullptr;  // 256 MiB written before each iteration in trace mode 2
    double stat_ms[amto::KSTAT_N] = {0, 0, 0};
    int stat_cnt[amto::KSTAT_N] = {0, 0, 0};
};

namespace amto {
// precompute.cu
// Dynamic shared memory of the pair kernel for a tile (n agents, nv
// coefficients, nb boundary rows, TC samples per unit, npad padded agents).
size_t pair_smem_bytes_host(int n, int nv, int nb, int TC, int npad, bool fused, int n_obs);
// Whether a plan with these parameters applies K^-1 inside the pair kernel.
bool apply_fused(const amto_params& p);
// Checks of amto_params (no CUDA call); sets the error text on failure.
amto_status validate_params(const amto_params& p);
amto_status precompute(amto_plan_s* pl);
// api.cu: a plan for validated parameters with shape choices of a batch of
// ref_batch (>= p.max_batch) instances; with a donor of the same parameters,
// its constants are taken over instead of recomputed (the donor is unchanged
// on failure).
amto_status create_plan(const amto_params& p, int ref_batch, bool tuned, amto_plan_s* donor,
                        amto_plan_s** out);
// A plan like `old` for new_batch (<= old's ref_batch) instances that takes
// over old's constants and the state of old's instances keep[0..nkeep)
// (ascending) as its instances 0..nkeep; the others start finished.  Runs on
// stream s and waits for it.  On success old keeps only its per-instance
// state (destroy it next); on failure old is unchanged.
amto_status plan_resize(amto_plan_s* old, int new_batch, const int* keep, int nkeep,
                        cudaStream_t s, amto_plan_s** out);
// Undo a resize: the constants go back from pl to old (which kept its
// state), and pl is freed.
void plan_give_back(amto_plan_s* pl, amto_plan_s* old);
// iterate.cu
amto_status configure_kernels(amto_plan_s* pl);
void gemm_workspace(const amto_plan_s* pl, size_t* ws_floats, int* tiles);
// `list` (device, nlist entries) restricts a launch to those instances of the
// plan's batch (continuous admission and retirement in the server).
amto_status launch_setup(amto_plan_s* pl, int batch, const float* start, const float* goal,
                         const float* bc_extra, const float* xi_init, int max_iters, float tol,
                         cudaStream_t s, const int* list = nullptr, int nlist = 0);
// init_mode 0: regular step; 1: initial projection, lambda = 0; 2: initial
// projection with lambda gathered from `lambda_init`.
amto_status launch_pair(amto_plan_s* pl, int batch, int init_mode, const float* lambda_init,
                        cudaGraphConditionalHandle h, int use_cond, cudaStream_t s,
                        const int* list = nullptr, int nlist = 0);
amto_status launch_rhs(amto_plan_s* pl, int batch, cudaStream_t s);
amto_status launch_apply(amto_plan_s* pl, int batch, cudaStream_t s);
amto_status launch_splitk_reduce(amto_plan_s* pl, int batch, int splits, cudaStream_t s);
// apply_tc.cu (tensor-core apply)
size_t tc_smem_bytes();
amto_status tc_configure(amto_plan_s* pl);
// Mixed batches (several plans iterated as one loop; csrc/mixed.cu).
amto_status launch_ctl_reset(Ctl* ctl, int max_iters, float tol, cudaStream_t s);
amto_status launch_rhs_mixed(amto_plan_s* const* pls, const int* batch, int ng, cudaStream_t s);
amto_status launch_mixed_cond(amto_plan_s* const* pls, int ng, Ctl* ctl,
                              cudaGraphConditionalHandle h, int use_cond, cudaStream_t s);
amto_status launch_apply_mixed(amto_plan_s* const* pls, const int* batch, int ng, cudaStream_t s);
amto_status configure_pair_mixed(amto_plan_s* const* pls, int ng, int* grid);
amto_status launch_pair_mixed(amto_plan_s* const* pls, const int* batch, int ng, Ctl* ctl,
                              int grid, cudaGraphConditionalHandle h, int use_cond,
                              cudaStream_t s);
// One-block-per-instance solver (csrc/block_solve.cu): the whole loop of
// every listed plan's batch in one launch (after setup and the initial
// projection, before the final residual).
size_t block_solver_smem(const PairGeom& g, int n, int m, int nv, int nb);
amto_status configure_block_solver(amto_plan_s* pl);
// Whether a plan with these parameters runs its loop in the block solver.
bool loop_block(const amto_params& p);
// AMTO_MULT_AUTO resolved: the aggregated multipliers where the reading and
// the loop allow them.
bool mult_aggregate(const amto_params& p);
// The autotuner's cached tile, apply and loop for p's shape (tune.cu): true
// and *out = p with those four fields set when p leaves all four automatic and
// a cached entry exists.
bool tune_lookup(const amto_params& p, amto_params* out);
// L = A_fc^T lambda_init of a warm start (AGGREGATE plans), one block per
// instance and axis.
amto_status launch_lambda_aggregate(amto_plan_s* pl, int batch, const float* lambda_init,
                                    cudaStream_t s);
amto_status launch_block_solver(amto_plan_s* const* pls, const int* batch, int ng, cudaStream_t s);
cudaError_t raise_smem_cap(const void* fn, size_t bytes);
// Tile grid, split-K count and K per split of the tensor-core apply.
void tc_shape(const amto_plan_s* pl, int batch, int* tm, int* tn, int* splits, int* kper);
// Kernel launches of one iteration of a batch-`batch` solve.
int launches_per_iteration(const amto_plan_s* pl, int batch);
amto_status launch_apply_tc(amto_plan_s* pl, int batch, cudaStream_t s);
amto_status launch_final(amto_plan_s* pl, int batch, float* xi_out, float* resid_out,
                         int* iters_out, cudaStream_t s, const int* list = nullptr, int nlist = 0);
// final_resid.cu: FP64 final residual of the lambda-free reading (unit skip,
// float-pair screen, FP64 confirmation of the candidates).
size_t final_free_smem(const amto_plan_s* pl);
// Screening chunks per instance of the final residual (lambda-free reading).
int final_free_ns(const PairGeom& g, int n, int m);
amto_status configure_final_free(amto_plan_s* pl);
amto_status launch_final_free(amto_plan_s* pl, int batch, cudaStream_t s, const int* list,
                              int nlist);
// Aggregated multipliers A_fc^T lambda of the last solve (user axes) / a
// warm start's into the plan (AGGREGATE plans).
amto_status launch_lagg_get(amto_plan_s* pl, int batch, float* out, cudaStream_t s);
amto_status launch_lagg_set(amto_plan_s* pl, int batch, const float* in, cudaStream_t s);
amto_status launch_state(amto_plan_s* pl, int batch, float* lambda_out, float* alpha_out,
                         float* beta_out, float* d_out, cudaStream_t s);
}  // namespace amto
