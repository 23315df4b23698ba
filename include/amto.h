/*
 * amto.h - C ABI of the B300 (sm_103a) alternating-minimisation multi-agent
 * trajectory optimiser of Rastgar et al., "GPU Accelerated Convex
 * Approximations for Fast Multi-Agent Trajectory Optimization" (arXiv
 * 2011.04240).
 *
 * The library computes Algorithm 1 of the paper: per iteration, the x/y/z
 * QPs (Eqs. step_x_3d-step_z_3d) through a cached inverse of the KKT matrix
 * (Eq. kkt_step_x, Remarks 1-2), the closed-form alpha/beta projection
 * (Eq. sphere_project), the d step clipped to d >= 1 (Eq. step_d and
 * Eq. alpha_beta_constr) and the multiplier update (Eq. lag_update), for a
 * batch of independent planning instances that share one agent count.
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  "device" pointers are CUDA device (or managed)
 *     memory of the current device; "host" pointers are ordinary host
 *     memory.  The caller owns every buffer it passes in; the plan owns its
 *     cached inverse and its workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous on it: outputs
 *     are valid once the stream has been synchronised.
 *   - No C++ exception and no abort crosses this boundary.  Every call
 *     returns an amto_status; amto_last_error() gives a thread-local text.
 *   - Agent-major layouts: xi is [batch][3 axes][n][deg+1] float32, with the
 *     Bernstein coefficients of agent i, axis ax at xi[(b*3+ax)*n*(deg+1) +
 *     i*(deg+1) + k] (the stacking c_x of Sec. III-B).
 *   - Pairs are the unordered pairs (i, j), i < j, numbered i-major
 *     (q = 0 for (0,1), 1 for (0,2), ...), the row order of Eq. (A_f);
 *     the pair difference is Delta = position_i - position_j.
 */
#ifndef AMTO_H
#define AMTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amto_plan_s* amto_plan;

typedef enum {
    AMTO_OK = 0,
    AMTO_EINVAL = 1,      /* invalid argument (message says which) */
    AMTO_ENOMEM = 2,      /* device or pinned-host allocation failed */
    AMTO_ECUDA = 3,       /* a CUDA runtime call failed */
    AMTO_ENONFINITE = 4,  /* non-finite input or state */
    AMTO_ETIMEOUT = 5,    /* a bounded device wait ran out */
    AMTO_ENUMERIC = 6,    /* the KKT inverse failed its self-check */
    AMTO_EPENDING = 7     /* a served request has not finished yet */
} amto_status;

/* Where lambda enters the alpha/beta/d steps (reading of Eqs. sphere_project
 * and step_d). */
enum {
    AMTO_PROJ_LITERAL = 0,  /* alpha, beta from Delta; d step with lambda^k / rho */
    AMTO_PROJ_NOLAMBDA = 1  /* lambda only in b_fc (Eq. b_f) and Eq. lag_update */
};

/* Arithmetic of the cached-inverse apply.  The pair projection is float32
 * in every mode. */
enum {
    AMTO_PREC_FP32 = 0,     /* float32 SIMT */
    AMTO_PREC_TF32X3 = 1,   /* tensor cores (tcgen05 kind::tf32): operands split into a
                               TF32 hi and a float32 lo part, 3 products (hi*hi + hi*lo +
                               lo*hi), float32 accumulate; tracks float32 to ~1e-6 */
    AMTO_PREC_BF16X3 = 2,   /* tensor cores (kind::f16, BF16 operands): BF16 hi and BF16
                               lo parts, 3 products, float32 accumulate (~16 bits) */
    AMTO_PREC_TF32 = 3,     /* tensor cores, TF32 operands, single product */
    AMTO_PREC_BF16 = 4,     /* tensor cores, BF16 operands, single product */
    /* Per-instance switch: the single product (TF32, or BF16) until the
     * instance's r_max stalls (it has not fallen below (1 - prec_drop) times
     * its best value within prec_window iterations), then the hi/lo
     * correction products as well (hi*lo + lo*hi, kept in a second
     * accumulator that only the switched instances add).  A tensor-core tile
     * whose instances have not switched skips the correction products.  The
     * switch is per instance and permanent for the solve; an instance's
     * arithmetic does not depend on the other instances of its batch. */
    AMTO_PREC_TF32_ADAPT = 5,
    AMTO_PREC_BF16_ADAPT = 6
};

/* Boundary-condition bits (rows of A in Sec. III-B). */
enum {
    AMTO_BC_POS0 = 1, AMTO_BC_VEL0 = 2, AMTO_BC_ACC0 = 4,
    AMTO_BC_POST = 8, AMTO_BC_VELT = 16, AMTO_BC_ACCT = 32,
    AMTO_BC_ALL = 63
};

typedef struct {
    int n_agents;      /* n, 2 <= n <= 256 */
    int m_steps;       /* samples per trajectory, poly_degree + 1 <= m <= 4096 */
    int poly_degree;   /* Bernstein degree N, 2 <= N <= 15 (N+1 coefficients) */
    double T;          /* horizon in seconds, > 0; samples t_k = k T / (m-1) */
    double a;          /* spheroid semi-axis l_xy, > 0 */
    double b;          /* spheroid semi-axis l_z, > 0 */
    double rho;        /* augmented-Lagrangian weight, > 0 */
    unsigned bc_mask;  /* AMTO_BC_* bits; must contain POS0 and POST */
    int proj_mode;     /* AMTO_PROJ_* */
    int precision;     /* AMTO_PREC_* */
    int max_batch;     /* largest batch a solve may take, >= 1 */
    /* Pair-kernel tiling (results do not depend on it; amto_tune measures):
     * agents per lane group (0 = automatic, else 8, 16 or 32) and time blocks
     * per warp and work unit (0 = automatic, else 1..8). */
    int tile_group;
    int tile_time_blocks;
    int apply_mode;    /* AMTO_APPLY_*: where the cached inverse is applied */
    int loop_mode;     /* AMTO_LOOP_*: how the iterations are driven */
    /* Increasing penalty (Sec. IV-A: several rho values, the larger ones in
     * later iterations; values and switch are this library's reading):
     * rho_j = rho * rho_growth^j for j < rho_stages, QP solve k >= 1 uses
     * stage min(rho_stages - 1, (k - 1) / rho_stage_iters), the multipliers
     * carry over.  One cached inverse per stage.  rho_stages 0 or 1: constant
     * rho.  A batch iterates in step (every instance of a solve is at the same
     * k), so the stages switch for the whole batch; the serving layer's slots
     * each follow their own (see amto_server_params). */
    int rho_stages;        /* 0..16 */
    double rho_growth;     /* > 0 when rho_stages > 1 */
    int rho_stage_iters;   /* >= 1 when rho_stages > 1 */
    int multipliers;       /* AMTO_MULT_*: how lambda is kept between iterations */
    /* Static obstacles per instance (Sec. IV-A: obstacles by their
     * circumscribing spheres, only the A_fc^T b_fc work grows with their
     * number): each (agent, obstacle, sample) is one more row of A_fc with a
     * fixed partner, the obstacle centre, projected on the combined
     * agent-obstacle spheroid given per obstacle (amto_set_obstacles).  The
     * penalty adds n_obstacles rho P^T P per agent to the KKT matrix, so the
     * cached inverse is the plan's.  0..64.  Plans with obstacles run the
     * graph loop with the batched, tensor-core or structured apply (not the
     * block solver, not the fused apply); mixed batches, the server and
     * amto_solve_static take plans without obstacles. */
    int n_obstacles;
    /* 1: agents are disks of radius l_xy in the x-y plane (Sec. III, "disks
     * in 2D"): alpha = atan2(Delta_y, Delta_x), u = l_xy (cos alpha,
     * sin alpha), Delta = 0 projects on +x; b (l_z) and every z input (start,
     * goal, boundary extras, warm starts, obstacle centres and l_z) are
     * ignored, and the returned z coefficients and multipliers are 0. */
    int planar;
    /* AMTO_PREC_*_ADAPT only: the stall test's window in iterations (0: 8)
     * and relative drop (0: 0.02); ignored by the other precisions. */
    int prec_window;
    double prec_drop;
} amto_params;

/* How the multipliers lambda (Eq. lag_update) are kept between iterations.
 * PAIRS: one float per pair, sample and axis, as Algorithm 1 keeps them;
 * every pair step reads and rewrites all of them (24 bytes per pair and
 * sample).  AGGREGATE (AMTO_PROJ_NOLAMBDA plans in the graph loop with the
 * batched or Kronecker apply): in that reading lambda enters an iteration
 * only through b_fc (Eq. b_f), and b_fc only through A_fc^T b_fc in the
 * right-hand side of Eq. kkt_step_x, which is linear in lambda; so the plan
 * keeps L = A_fc^T lambda (3 n (N+1) floats per instance) and updates it with
 * the same linear map, L_k = L_{k-1} + rho_k A_fc^T f_c^k.  The iterates are
 * those of PAIRS in exact arithmetic (float32 rounding differs), and the
 * pair step then reads and writes no per-pair state.  The per-pair
 * multipliers of such a plan are never formed: amto_get_state returns
 * EINVAL for lambda_out (alpha, beta and d, which this reading computes
 * from Delta alone, are still returned).  A warm start's lambda_init is
 * reduced to L once, in the solve's setup.  AUTO: AGGREGATE where allowed,
 * else PAIRS. */
enum { AMTO_MULT_AUTO = 0, AMTO_MULT_PAIRS = 1, AMTO_MULT_AGGREGATE = 2 };

/* How the loop of Algorithm 1 runs.  GRAPH: one CUDA graph per batch size,
 * a conditional WHILE node around the iteration's kernels (right-hand side,
 * apply, pair step), every instance of the batch in every launch.  BLOCK
 * (float32, batched apply): one thread block per instance runs the whole
 * loop (right-hand side, K^-1 matrix-vector product from L2, pair step, the
 * stopping rule) with no launch between iterations; for small instances and
 * latency-bound solves.  AUTO: BLOCK for float32 plans with n_agents <= 8
 * and max_batch <= 148 (one wave of blocks), else GRAPH (measured crossover
 * on B300; amto_tune measures both). */
enum { AMTO_LOOP_AUTO = 0, AMTO_LOOP_GRAPH = 1, AMTO_LOOP_BLOCK = 2 };

/* Where the step xi += K^-1_top [g; e] runs.  BATCHED: a separate right-hand-
 * side launch and one GEMM launch over the batch per iteration (tensor cores
 * in the TF32/BF16 modes).  FUSED (float32 only): the last block of each
 * instance's pair step forms its right-hand side and applies K^-1 as a
 * matrix-vector product (K^-1 read from L2), so an iteration is one launch.
 * AUTO: BATCHED (faster on B300 at every size measured; amto_tune measures
 * both).  KRONECKER (any precision; the apply itself is float32): the exact
 * agent structure of the inverse, K^-1 = I (x) K_n^-1 + (1/n) 1 1^T (x)
 * (K_0^-1 - K_n^-1) with K_n, K_0 the agent-level KKT matrices with
 * smoothness plus rho n P^T P and smoothness only, applied as
 * xi_i += K_n^-1_top (r_i - r_mean) + K_0^-1_top r_mean: O(17^2 n) per axis
 * instead of the dense O(187 n^2); the same result in exact arithmetic,
 * not the paper's dense product (a variant, measured against it). */
enum {
    AMTO_APPLY_AUTO = 0,
    AMTO_APPLY_BATCHED = 1,
    AMTO_APPLY_FUSED = 2,
    AMTO_APPLY_KRONECKER = 3
};

typedef struct {
    int n_agents, m_steps, nv, nb;      /* nv = N+1 coefficients, nb = #BC rows */
    int kkt_dim;                        /* (nv + nb) * n */
    int group;                          /* agents per lane group of the pair kernel */
    int t_chunk;                        /* time samples per pair-kernel work unit */
    int n_chunks;                       /* pair-kernel work units per instance */
    long long lambda_floats;            /* float32 multiplier slots per instance (one buffer;
                                           0 for AMTO_MULT_AGGREGATE plans) */
    double kkt_check;                   /* max |K K^-1 - I| of the FP64 inverse */
    size_t device_bytes;                /* device memory owned by the plan */
    int launches_per_iteration;         /* kernels per iteration at batch = max_batch:
                                           right-hand side, apply (+ split-K reduce),
                                           pair step */
    int launches_fixed;                 /* kernels per solve outside the loop: setup,
                                           initial projection, FP64 residual (three
                                           in the lambda-free reading: unit bounds,
                                           screen, confirmation), outputs (+1: block
                                           solver) */
    int time_blocks;                    /* pair-kernel time blocks per warp and unit */
    int apply_mode;                     /* AMTO_APPLY_BATCHED, _FUSED or _KRONECKER */
    int loop_mode;                      /* AMTO_LOOP_GRAPH or AMTO_LOOP_BLOCK */
    int multipliers;                    /* AMTO_MULT_PAIRS or AMTO_MULT_AGGREGATE */
    int n_obstacles;                    /* static obstacles per instance */
    int planar;                         /* 1: disks in the x-y plane */
    int tuned;                          /* 1: tile, apply and loop came from the
                                           autotuner's cache (see amto_tune) */
} amto_info;

/*
 * amto_create - build a plan for one agent count (Remarks 1-2: the KKT
 * matrix depends on n, rho and the basis only, so its inverse is computed
 * once and reused for any start/goal).
 *
 * On the current CUDA device: forms the Bernstein basis P, Pdot, Pddot
 * (Eq. param), Q_x, A, A_eq and the KKT matrix of Eq. (kkt_step_x), forms
 * its inverse in FP64 from the exact agent-level closed form
 * K^-1 = I (x) K_n^-1 + (1/n) 1 1^T (x) (K_0^-1 - K_n^-1) (two small
 * agent-level KKT matrices inverted by Gauss-Jordan elimination with partial
 * pivoting), checks max|K K^-1 - I| against K assembled from its
 * definition, and keeps the top block rows of the inverse in float32.
 * Allocates all device workspace for `max_batch` instances, so amto_solve
 * allocates nothing.  Synchronous.  Errors: EINVAL for out-of-range
 * params, ENOMEM, ECUDA, ENUMERIC if the inverse fails its self-check.
 * *out is NULL on error.
 */
amto_status amto_create(const amto_params* params, amto_plan* out);

/* Release the plan and all device memory it owns.  NULL is a no-op.
 * Synchronises the device work the plan issued. */
void amto_destroy(amto_plan plan);

/*
 * amto_solve - run Algorithm 1 on `batch` instances (1 <= batch <= max_batch).
 *
 *   start, goal  device [batch][n][3] float32: positions at t = 0 and t = T
 *                (b_eq of Sec. III-B).
 *   bc_extra     device [batch][n][2][2][3] float32 or NULL: [t0 | T]
 *                [velocity | acceleration][axis] boundary values (zero when
 *                NULL).
 *   xi_init      device [batch][3][n][N+1] float32 or NULL: warm-start
 *                trajectories; NULL = smoothness-only initialisation.
 *   lambda_init  device [batch][3][p][m] float32 or NULL (p = n(n-1)/2,
 *                pair-major then time): warm-start multipliers; NULL = 0.
 *   max_iters    >= 0 iterations (QP solves) at most.
 *   tol          stop an instance once its max over pairs and samples of
 *                ||f_c||_2 (Eq. sphere_proposed) is below tol after at
 *                least one iteration; 0 = run max_iters.
 *   xi_out       device [batch][3][n][N+1] float32: final trajectories.
 *   resid_out    device [batch] float32 or NULL: final max ||f_c||_2,
 *                recomputed in FP64 from the final trajectories and
 *                multipliers; NaN for an instance with non-finite input.
 *   iters_out    device [batch] int32 or NULL: iterations performed; -1 for
 *                an instance with non-finite input or state.
 *
 * The whole iteration loop runs on the device (a CUDA graph with a
 * device-side loop condition); nothing is allocated after the first solve
 * of a given batch size (which instantiates that graph).  Errors: EINVAL
 * (sizes, NULL required pointers), ECUDA.  Non-convergence is not an
 * error: iters_out = max_iters and the residual is reported.
 */
amto_status amto_solve(amto_plan plan, int batch,
                       const float* start, const float* goal, const float* bc_extra,
                       const float* xi_init, const float* lambda_init,
                       int max_iters, float tol,
                       float* xi_out, float* resid_out, int* iters_out,
                       void* stream);

/*
 * amto_solve_static - the solve of amto_solve for ONE instance (batch 1, no
 * boundary extras, no warm start) that allocates no memory at all.  The
 * paper has no counterpart; this is a library convenience.
 *
 * For callers that cannot call cudaMalloc while they plan: a control loop
 * with a fixed memory budget, a process whose device heap is owned by its
 * own pool allocator, or a thread that must not take the allocator's locks.
 * All per-solve buffers (trajectories, boundary values, both multiplier
 * buffers, partial sums, right-hand side, flags) come from one static device
 * array of 8 MiB that every GPU loading this library holds until the
 * process exits.  The plan's read-only constants, made by amto_create, are
 * reused.  A plan whose one-instance buffers do not fit in 8 MiB (about
 * n > 80 agents at m = 100) is rejected with AMTO_EINVAL and a message
 * giving the bytes it would need.
 *
 *   start, goal  device [1][n][3] float32;  xi_out device [1][3][n][N+1];
 *   resid_out, iters_out as in amto_solve (device, may be NULL).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and keeps it for that
 * device's CUDA context; make that first call before any stream capture on
 * the device.  A new context on the device (after cudaDeviceReset) is
 * noticed by its context id and the address looked up again on the next
 * call.  Every call shares the one array and overwrites it; the flags and
 * counters that must start at zero are cleared by each call.  Calls that
 * overlap on the GPU (for example on two streams) race on the array:
 * serialise them.
 *
 * The loop is driven from the host: it launches one iteration's kernels
 * (right-hand side, the matrix-vector apply, pair step) per pass and
 * synchronises `stream` every 8 passes to read the stop flag, so up to 7
 * passes may be launched after every instance has stopped; the device
 * control block marks the instance done and those passes do no work.
 * Because it always uses the graph loop's kernels with the one-instance
 * matrix-vector apply, its trajectories match amto_solve's on the same
 * plan and inputs within the float32 tolerance of the parity tests (a plan
 * whose amto_solve runs the batched split-K product or the one-block loop
 * sums in another order), and near `tol` the iteration count may differ.
 * Errors: EINVAL, ECUDA.
 */
amto_status amto_solve_static(amto_plan plan, const float* start, const float* goal,
                              int max_iters, float tol, float* xi_out, float* resid_out,
                              int* iters_out, void* stream);

/*
 * amto_get_aggregate - the multipliers of the last solve on an
 * AMTO_MULT_AGGREGATE plan, in the form the plan keeps them: A_fc^T lambda
 * (Eq. A_f's transpose applied to the lambda of Eq. lag_update), the
 * per-agent, per-coefficient sum of every pair's multiplier times its
 * basis row with the pair's sign (+ for the first agent of a pair, - for
 * the second), after the last solve's final update (lambda^K for K
 * iterations; the warm-start value for K = 0).
 *
 *   agg_out  device [batch][3][n][N+1] float32 (written; caller-owned).
 *
 * `batch` must equal the last solve's batch.  Asynchronous on `stream`.
 * Errors: EINVAL (NULL pointers, batch, or a plan that keeps lambda per
 * pair: read those with amto_get_state).  Together with the returned
 * trajectories this is the state that amto_solve_from_aggregate resumes from.
 */
amto_status amto_get_aggregate(amto_plan plan, int batch, float* agg_out, void* stream);

/*
 * amto_solve_from_aggregate - amto_solve on an AMTO_MULT_AGGREGATE plan
 * with warm-start multipliers given in aggregated form: agg_init (device
 * [batch][3][n][N+1] float32, caller-owned, read before the call's kernels
 * finish) is A_fc^T lambda, as amto_get_aggregate returns it; it is
 * equivalent to passing the per-pair lambda it was formed from as
 * amto_solve's lambda_init.  Every other argument is amto_solve's; xi_init
 * is usually the trajectories the state was read with.  Errors: EINVAL
 * (also for a plan that keeps lambda per pair), ECUDA.
 */
amto_status amto_solve_from_aggregate(amto_plan plan, int batch, const float* start,
                                      const float* goal, const float* bc_extra,
                                      const float* xi_init, const float* agg_init,
                                      int max_iters, float tol, float* xi_out,
                                      float* resid_out, int* iters_out, void* stream);

/*
 * amto_get_state - read back the multipliers of the last solve on this plan
 * and alpha, beta, d of its last projection (Eqs. sphere_project, step_d).
 * All outputs are device pointers, each may be NULL:
 *   lambda_out [batch][3][p][m], alpha_out/beta_out/d_out [batch][p][m],
 * float32.  `batch` must equal the last solve's batch.  Asynchronous.
 * EINVAL if lambda_out is given for an AMTO_MULT_AGGREGATE plan.
 */
amto_status amto_get_state(amto_plan plan, int batch, float* lambda_out,
                           float* alpha_out, float* beta_out, float* d_out,
                           void* stream);

/*
 * amto_set_obstacles - the static obstacles of instances 0..batch-1 for the
 * plan's later solves (reading R-obst): device array [batch][n_obstacles][5]
 * of float32 (centre x, y, z, then the semi-axes l_xy, l_z of the combined
 * agent-obstacle spheroid, e.g. agent half-extent plus obstacle radius).
 * Copied asynchronously on `stream` into the plan (the caller may reuse the
 * array once the stream has passed this call).  A solve of a plan with
 * obstacles needs them set for all of its instances (else EINVAL); an
 * instance with a non-finite value or a semi-axis <= 0 is flagged non-finite
 * by the solve (residual NaN, iterations -1).  lambda_init of a warm start
 * covers the pairs only; the obstacle multipliers start at 0.  EINVAL if the
 * plan has no obstacles or batch is outside [1, max_batch].
 */
amto_status amto_set_obstacles(amto_plan plan, int batch, const float* obstacles, void* stream);

/* Sizes and self-check figures of a plan (host struct, synchronous). */
amto_status amto_get_info(amto_plan plan, amto_info* out);

/*
 * amto_get_kkt_inverse - copy the FP64 KKT inverse, (nv+nb)n x (nv+nb)n
 * row-major, unknowns ordered [c (agent-major) ; multipliers (agent-major)],
 * to host memory `out` (kkt_dim^2 doubles).  Synchronous.
 */
amto_status amto_get_kkt_inverse(amto_plan plan, double* out);

/*
 * amto_get_stats - per-kernel device time of the most recent traced solve
 * (see amto_set_trace): out_ms[k] total milliseconds and out_count[k]
 * launches for k = 0 pair kernel, 1 rhs kernel, 2 apply kernel.  Host
 * arrays of length 3.
 */
amto_status amto_get_stats(amto_plan plan, double* out_ms, int* out_count);

/*
 * amto_set_trace - 1: later solves launch each kernel from a host loop and
 * bracket it with CUDA events on the solve's stream (per-kernel timing, no
 * graph, one host synchronisation per iteration); 2: as 1, and before each
 * iteration the L2 cache is flushed by writing a 256 MiB device buffer (taken
 * by this call, freed with the plan), outside the timed events, so every
 * iteration's kernels start from HBM; 0: graph mode (default).  Results are
 * identical in all modes.  ENOMEM if the flush buffer cannot be allocated.
 */
amto_status amto_set_trace(amto_plan plan, int on);

/* ------------------------------------------------------------------------
 * Autotuning of the pair-kernel tile (the library's own; the paper has no
 * counterpart).  The tile (tile_group, tile_time_blocks of amto_params)
 * changes which lanes and blocks process which pairs and samples, never a
 * result.
 * ------------------------------------------------------------------------ */
#define AMTO_TUNE_MAX 48

typedef struct {
    int tile_group;            /* agents per lane group: 8, 16 or 32 */
    int tile_time_blocks;      /* time blocks per warp and work unit */
    int apply_mode;            /* AMTO_APPLY_BATCHED or AMTO_APPLY_FUSED */
    int loop_mode;             /* AMTO_LOOP_GRAPH or AMTO_LOOP_BLOCK */
    double us_per_iteration;   /* measured loop time per iteration of the batch */
} amto_tune_entry;

typedef struct {
    int n_entries;
    amto_tune_entry entries[AMTO_TUNE_MAX];  /* every candidate measured, in order */
    int best;                                /* index of the fastest entry */
} amto_tune_result;

/* Measure every tile (and, for float32 plans, the apply and loop modes) that
 * fits `params` (its tile, apply_mode and loop_mode fields are ignored) on a
 * synthetic batch of `batch` instances (agents on a ring, antipodal goals),
 * `iters` fixed iterations each: a plan per candidate is created, solved
 * twice (2 and 2 + iters iterations, the difference is the loop time) and
 * destroyed.  Synchronous; uses the current device.  The best entry is kept
 * in the tuning cache (below), so that later plans of this shape with an
 * automatic tile use it; its four fields can also be copied into amto_params.
 * Errors: EINVAL (bad params, 1 <= batch <= max_batch, 1 <= iters <= 1e5),
 * ENOMEM, ECUDA. */
amto_status amto_tune(const amto_params* params, int batch, int iters, amto_tune_result* out);

/* The tuning cache.  amto_tune keeps its best entry in a process-wide cache
 * under the key (n_agents, m_steps, poly_degree, batch rounded up to a power
 * of two, precision, proj_mode, multipliers, n_obstacles, planar, rho_stages,
 * bc_mask); a later entry of the same key replaces the earlier one.
 * amto_create (and so the mixed batches and the server, which create their
 * plans through it) takes the cached tile, apply and loop for a plan of the
 * same key (max_batch rounded up the same way) whose tile_group,
 * tile_time_blocks, apply_mode and loop_mode are all 0 (automatic), as long as
 * the choice is valid for its parameters; amto_info.tuned reports it.
 * save writes one text line per entry ("amto-tune-v1" and 17 fields); load
 * merges a file written by save into the cache (EINVAL, nothing merged, on an
 * unreadable file or a malformed line).  Thread-safe. */
amto_status amto_tune_cache_save(const char* path);
amto_status amto_tune_cache_load(const char* path);
void amto_tune_cache_clear(void);
int amto_tune_cache_size(void);

/* ------------------------------------------------------------------------
 * Mixed batches: instances with different agent counts iterated as one loop.
 *
 * The paper solves one problem (one agent count) at a time; grouping several
 * plans is the library's own.  Every plan keeps its cached inverse (Remarks
 * 1-2: it depends on the agent count only) and its state for up to max_batch
 * instances.  Per iteration one launch forms the right-hand sides of all
 * instances, one launch runs the cached-inverse GEMM tiles of all FP32 plans
 * (tensor-core plans run their own apply), and one persistent launch runs the
 * pair step (Algorithm 1's projection, multiplier update and A_fc^T
 * reduction) for the (instance, time-chunk) units of all plans; the loop is a
 * CUDA graph under a conditional WHILE node (built once per combination of
 * batch sizes), stopping when no instance of any plan is still iterating.
 * Per instance the result is that of amto_solve on its own plan (same
 * arithmetic; only the launches are shared).  The layout (below) chooses
 * between one fused launch over all plans and per-plan parallel branches.
 * ------------------------------------------------------------------------ */
#define AMTO_MAX_MIXED_GROUPS 8

/* Layout of a mixed iteration.  FUSED: one right-hand-side launch, one
 * grouped apply and one persistent pair-step launch over the units of all
 * plans.  BRANCHES: every plan's own chain (right-hand side, apply, pair
 * step) as a parallel branch of the graph body, joined by one kernel that
 * sets the loop condition, so different agent counts overlap on the device.
 * LOOPS: every plan's own loop (its own conditional WHILE node over its
 * chain, its own stopping count) as a parallel branch of one graph, joined
 * only when all have finished: no count waits for another between
 * iterations.  With LOOPS each plan's penalty schedule follows its own pass
 * count, as in its own solve. */
enum { AMTO_MIXED_FUSED = 0, AMTO_MIXED_BRANCHES = 1, AMTO_MIXED_LOOPS = 2 };

typedef struct amto_mixed_s* amto_mixed;

/* Group n_plans (1..AMTO_MAX_MIXED_GROUPS) distinct plans that agree on
 * device, m_steps, poly_degree, T, a, b, rho, bc_mask and proj_mode.  The
 * plans must outlive the mixed object, and a plan must not be solved by
 * another call while a mixed solve that uses it is in flight.
 * Errors: EINVAL, ENOMEM, ECUDA. */
amto_status amto_mixed_create(const amto_plan* plans, int n_plans, int layout, amto_mixed* out);

/* Solve batch[g] instances with plan g, for every g, as one loop; arguments
 * per group are as in amto_solve (all six boundary conditions from start and
 * goal with zero end velocities and accelerations, no warm start):
 *   batch      host [n_plans], 1 <= batch[g] <= max_batch of plan g
 *   start[g], goal[g]  device [batch[g]][n_g][3]   (host arrays of pointers)
 *   xi_out[g]  device [batch[g]][3][n_g][N+1]; resid_out[g], iters_out[g]
 *              device [batch[g]] (the arrays or entries may be NULL)
 * Asynchronous on `stream`.  Errors: EINVAL, ECUDA. */
amto_status amto_mixed_solve(amto_mixed mixed, const int* batch, const float* const* start,
                             const float* const* goal, int max_iters, float tol,
                             float* const* xi_out, float* const* resid_out,
                             int* const* iters_out, void* stream);

/* 1: run the loop from the host, one launch at a time (what profilers need;
 * identical results), 0: the graph loop (default). */
amto_status amto_mixed_set_trace(amto_mixed mixed, int on);

void amto_mixed_destroy(amto_mixed mixed);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of requests of mixed agent counts.
 *
 * The paper solves one problem at a time; this serving layer is the library's
 * own.  A server keeps one plan per served agent count (the cached inverse of
 * Remarks 1-2 is shared by all requests of that count) with a number of
 * resident instance slots fixed by a device-memory budget.  A worker thread
 * admits queued requests into free slots between iteration chunks while the
 * other slots keep iterating, runs each agent count's resident slots as one
 * batched step (one GEMM with the cached inverse per count and iteration; the
 * counts on separate streams, overlapping on the device), and retires
 * instances whose stopping rule fired.  A request's result does not depend
 * on the other requests in flight.
 * ------------------------------------------------------------------------ */
typedef struct amto_server_s* amto_server;

typedef struct {
    int n_sizes;           /* number of served agent counts, 1..32 */
    const int* sizes;      /* host [n_sizes] distinct agent counts */
    int m_steps, poly_degree;
    double T, a, b, rho;   /* as in amto_params; all six boundary conditions */
    int proj_mode, precision;
    int max_slots;         /* upper bound on resident instances per agent count */
    int chunk_iters;       /* iterations between admission / retirement points */
    int max_iters;         /* per-request iteration cap */
    float tol;             /* per-request stopping tolerance on max ||f_c|| */
    size_t memory_budget;  /* device bytes for resident per-instance state (xi, multipliers,
                              partial sums, right-hand sides); 0 = half the free memory.
                              Each agent count starts with an equal share (its fair
                              share): as many slots as instances whose state fits in
                              it, at most max_slots.  See `admission` for how the
                              shares then move.  Each count's cached inverse and the
                              plan's fixed buffers come on top of the budget. */
    /* Increasing rho per request (as amto_params; 0 or 1: constant rho).  The
     * slots are not in step, so each request follows the schedule from its
     * own QP count; the server then applies K^-1 in its structured form
     * (AMTO_APPLY_KRONECKER), whose stage is chosen per instance. */
    int rho_stages;
    double rho_growth;
    int rho_stage_iters;
    /* AMTO_ADMIT_SHARED (0, default): one budget for all counts.  Between
     * chunks, the count with the most queued requests beyond its free slots
     * doubles its slot capacity (up to max_slots or the whole budget), from
     * unclaimed budget and by shrinking other counts: an idle count (empty
     * queue) down to max(min(8, its fair share), the next power of two >= its
     * resident instances), a count with a queue never below its fair share.
     * A count grows, and a donor shrinks, by a quarter of its capacity or more.
     * While a count waits below its fair share, counts above theirs admit no
     * new requests beyond it.  A resize moves the resident instances' state to
     * a plan of the new capacity (the cached inverse is taken over, not
     * recomputed); their results do not change, because every shape choice
     * (lane group, the apply's split over K) is fixed at creation by the
     * largest capacity the count can reach.  During a resize the count's old
     * and new state exist side by side for a moment.
     * AMTO_ADMIT_FIXED (1): every count keeps its fair share. */
    int admission;
} amto_server_params;

enum { AMTO_ADMIT_SHARED = 0, AMTO_ADMIT_FIXED = 1 };

typedef struct {
    int n_agents;          /* must be one of the served counts */
    const float* start;    /* host [n][3]; copied by amto_server_submit */
    const float* goal;     /* host [n][3] */
} amto_request;

typedef struct {
    int iters;             /* iterations performed (-1: non-finite input or state;
                              -2: a bounded wait in the iteration kernel gave up) */
    float resid;           /* final max ||f_c||, recomputed in FP64 */
    double t_submit, t_admit, t_done;  /* seconds on a monotonic clock */
} amto_result_info;

typedef struct {
    long long completed, iterations, chunks;
    int n_groups;
    int sizes[32], slots[32];  /* served counts and their current slot capacities */
    int fair_slots[32];        /* each count's fair share of the budget, in slots */
    int max_capacity[32];      /* the largest capacity each count may reach */
    long long resizes;         /* capacity changes so far (AMTO_ADMIT_SHARED) */
    size_t budget, budget_used;  /* the memory budget and the bytes the slots hold */
} amto_server_stats_t;

/* Create a server and start its worker thread on the current device.
 * Errors: EINVAL, ENOMEM (budget too small for one instance), ECUDA. */
amto_status amto_server_create(const amto_server_params* params, amto_server* out);

/* Queue one request (inputs are copied; non-blocking).  *ticket identifies it. */
amto_status amto_server_submit(amto_server server, const amto_request* req, uint64_t* ticket);

/* Collect a finished request: waits up to wait_ms for it, then returns
 * AMTO_EPENDING if it is still running, or its status (AMTO_OK, ENONFINITE, ETIMEOUT)
 * after copying xi (host [3][n][N+1], may be NULL) and *info (may be NULL).
 * A collected ticket is forgotten. */
amto_status amto_server_poll(amto_server server, uint64_t ticket, int wait_ms, float* xi_out,
                             amto_result_info* info);

/* One step of the shared-budget admission policy (AMTO_ADMIT_SHARED) on a
 * description of the served counts, with no device work: the server applies
 * the same step between chunks.  Inputs per count (host arrays of n_counts,
 * 1..32): slot capacity, resident requests (<= slots), queued requests, fair
 * share and largest capacity in slots (slots <= max_capacity <= 65535), and
 * device bytes per resident instance; budget in bytes.  slots_out (host
 * [n_counts]) receives the capacities after the step (unchanged counts keep
 * theirs).  Errors: EINVAL. */
amto_status amto_admission_step(int n_counts, const int* slots, const int* active,
                                const int* queued, const int* fair_slots, const int* max_capacity,
                                const unsigned long long* bytes_per_instance,
                                unsigned long long budget, int* slots_out);

/* Counters of the server (completed requests and their iterations, chunks). */
amto_status amto_server_stats(amto_server server, amto_server_stats_t* out);

/* Stop the worker (requests still queued are dropped) and free everything. */
void amto_server_destroy(amto_server server);

/* Thread-local text of the last error on this thread ("" if none). */
const char* amto_last_error(void);

/* Library version string. */
const char* amto_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AMTO_H */
