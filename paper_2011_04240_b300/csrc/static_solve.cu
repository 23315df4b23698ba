// amto_solve_static: a solve of one instance that allocates nothing.
//
// Some callers cannot allocate device memory at solve time: code that runs
// inside a real-time control loop with a fixed memory budget, callers that
// own the whole device heap through their own pool, or callers whose
// allocator is not allowed to be touched from the planning thread.  For them
// this entry point runs the same kernels as amto_solve (batch of one, no warm
// start) but takes every per-solve buffer (trajectory state, boundary
// values, both multiplier buffers, partial sums, right-hand side, flags,
// control block) from one file-scope device array of fixed size instead of
// the plan's workspace.  The plan's read-only constants (the cached KKT
// inverse, the basis) are still used; they were allocated when the plan was
// created.  The iteration loop is driven from the host and checks the
// device-side stop flag every few iterations with a plain copy to host stack
// memory.  This file has no counterpart in the paper.
#include <cmath>
#include <cstring>
#include <mutex>

#include "amto_internal.cuh"

namespace amto {
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kPollEvery = 8;  // iterations between host checks of the stop flag

// Held by every GPU that loads the library until the process exits.  In host
// code the name is only a stand-in for the symbol; kernels get the device
// address obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context id the address belongs to

// Id of the calling thread's current CUDA context (unique for the process's
// lifetime, so a context made after cudaDeviceReset has a new one); 0 when
// the driver does not provide it, in which case nothing is cached.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on `dev` (the current device).  It is
// looked up with cudaGetSymbolAddress on the first call in a context and kept
// for that context: a device reset makes a new context, whose id differs, and
// the address is looked up again (the module and its array may have moved).
amto_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("amto_solve_static: device ordinal out of range");
        return AMTO_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("amto_solve_static: cudaGetSymbolAddress failed: ") +
                      cudaGetErrorString(e));
            return AMTO_ECUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return AMTO_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace amto

using namespace amto;

extern "C" amto_status amto_solve_static(amto_plan plan, const float* start, const float* goal,
                                         int max_iters, float tol, float* xi_out,
                                         float* resid_out, int* iters_out, void* stream) {
    clear_error();
    if (!plan) {
        set_error("invalid argument: plan is NULL");
        return AMTO_EINVAL;
    }
    if (plan->prm.n_obstacles > 0) {
        set_error("invalid argument: amto_solve_static takes plans without obstacles");
        return AMTO_EINVAL;
    }
    if (plan->prm.precision != AMTO_PREC_FP32) {
        set_error("invalid argument: amto_solve_static takes plans made with AMTO_PREC_FP32");
        return AMTO_EINVAL;
    }
    if (!start || !goal || !xi_out) {
        set_error("invalid argument: start, goal and xi_out are required");
        return AMTO_EINVAL;
    }
    if (max_iters < 0 || !(tol >= 0.f) || !(tol < INFINITY)) {
        set_error("invalid argument: max_iters must be >= 0 and tol a finite value >= 0");
        return AMTO_EINVAL;
    }
    const amto_plan_s& pl = *plan;
    const size_t nvn = (size_t)pl.n * pl.nv, NC = pl.geo.n_chunks;
    // carve the per-solve buffers of one instance out of the scratch array
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += align256(bytes);
        return at;
    };
    const size_t o_xi = take(sizeof(float) * 3 * nvn);
    const size_t o_beq = take(sizeof(float) * 3 * pl.n * pl.nb);
    const size_t lam_b = pl.agg ? 0 : sizeof(float) * (size_t)pl.geo.lam_floats;
    const size_t o_lam0 = take(lam_b);
    const size_t o_lam1 = take(lam_b);
    const size_t o_lagg = take(pl.agg ? sizeof(float) * 3 * nvn : 0);
    const size_t o_gpart = take(sizeof(float) * NC * 3 * nvn);
    const size_t o_rpart = take(sizeof(float) * NC);
    const size_t o_spart = take(sizeof(float) * NC);
    const size_t NSf = (size_t)final_free_ns(pl.geo, pl.n, pl.m);
    const size_t o_fin = take(sizeof(float) * NSf * kFinRecFloats);
    const size_t o_fwork = take(sizeof(int) * NSf);
    const size_t o_fctl = take(sizeof(unsigned) * 2);
    const size_t o_folim = take(sizeof(float));
    const size_t o_rhs = take(sizeof(float) * 3 * (size_t)pl.kp);
    const size_t o_rmax = take(sizeof(float));
    const size_t o_r64 = take(sizeof(unsigned long long));
    const size_t o_iters = take(sizeof(int));
    const size_t o_flags = take(sizeof(int));
    const size_t o_tk = take(sizeof(unsigned));
    const size_t o_ctl = take(sizeof(Ctl));
    if (off > kStaticScratchBytes) {
        set_error("invalid argument: amto_solve_static needs " + std::to_string(off) +
                  " bytes of scratch for this plan but the static array holds " +
                  std::to_string(kStaticScratchBytes) + " bytes; use amto_solve");
        return AMTO_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != pl.device && cudaSetDevice(pl.device) != cudaSuccess) {
        set_error("amto_solve_static: cannot select the plan's device");
        return AMTO_ECUDA;
    }
    struct Restore {
        int dev, plan_dev;
        ~Restore() {
            if (dev >= 0 && dev != plan_dev) cudaSetDevice(dev);
        }
    } restore{prev, pl.device};
    unsigned char* base = nullptr;
    amto_status st = scratch_address(pl.device, &base);
    if (st != AMTO_OK) return st;

    // a view of the plan whose workspace pointers point into the scratch
    amto_plan_s v;
    v.prm = pl.prm;
    v.prm.max_batch = 1;  // one instance: the apply runs as the matrix-vector kernel
    v.ref_batch = 1;
    v.device = pl.device;
    v.num_sms = pl.num_sms;
    v.n = pl.n; v.m = pl.m; v.N = pl.N; v.nv = pl.nv; v.nb = pl.nb; v.kdim = pl.kdim; v.p = pl.p;
    v.geo = pl.geo;
    v.P32 = pl.P32; v.P64 = pl.P64; v.Q32 = pl.Q32; v.A32 = pl.A32; v.E0 = pl.E0;
    v.Kinv64 = pl.Kinv64; v.Ktop = pl.Ktop; v.kp = pl.kp;
    v.fused = pl.fused;
    v.kron = pl.kron;
    v.Kag = pl.Kag;
    v.sched = pl.sched;
    v.ks_top = pl.ks_top; v.ks_ag = pl.ks_ag;
    v.xi = reinterpret_cast<float*>(base + o_xi);
    v.beq = reinterpret_cast<float*>(base + o_beq);
    v.agg = pl.agg;
    v.lam[0] = pl.agg ? nullptr : reinterpret_cast<float*>(base + o_lam0);
    v.lam[1] = pl.agg ? nullptr : reinterpret_cast<float*>(base + o_lam1);
    v.Lagg = pl.agg ? reinterpret_cast<float*>(base + o_lagg) : nullptr;
    v.gpart = reinterpret_cast<float*>(base + o_gpart);
    v.rpart = reinterpret_cast<float*>(base + o_rpart);
    v.spart = reinterpret_cast<float*>(base + o_spart);
    v.fin = reinterpret_cast<float*>(base + o_fin);
    v.fin_work = reinterpret_cast<int*>(base + o_fwork);
    v.fin_ctl = reinterpret_cast<unsigned*>(base + o_fctl);
    v.fin_olim = reinterpret_cast<float*>(base + o_folim);
    v.fin_grid = pl.fin_grid;
    v.P32lo = pl.P32lo;
    v.rhs = reinterpret_cast<float*>(base + o_rhs);
    v.rmax = reinterpret_cast<float*>(base + o_rmax);
    v.r64 = reinterpret_cast<unsigned long long*>(base + o_r64);
    v.iters = reinterpret_cast<int*>(base + o_iters);
    v.flags = reinterpret_cast<int*>(base + o_flags);
    v.uticket = reinterpret_cast<unsigned*>(base + o_tk);
    v.ctl = reinterpret_cast<Ctl*>(base + o_ctl);

    cudaStream_t s = (cudaStream_t)stream;
    // k_setup clears the flags, counters, tickets and control block that must
    // start at zero; the initial projection writes the first multiplier buffer.
    st = launch_setup(&v, 1, start, goal, nullptr, nullptr, max_iters, tol, s);
    if (st == AMTO_OK) st = launch_pair(&v, 1, 1, nullptr, 0, 0, s);
    for (int it = 0; st == AMTO_OK && it <= max_iters; ++it) {
        if (it % kPollEvery == 0) {
            Ctl c;
            if (cudaMemcpyAsync(&c, v.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                set_error("amto_solve_static: reading the stop flag failed");
                return AMTO_ECUDA;
            }
            if (c.active_last == 0) break;
        }
        st = launch_rhs(&v, 1, s);
        if (st == AMTO_OK) st = launch_apply(&v, 1, s);
        if (st == AMTO_OK) st = launch_pair(&v, 1, 0, nullptr, 0, 0, s);
    }
    if (st == AMTO_OK) st = launch_final(&v, 1, xi_out, resid_out, iters_out, s);
    return st;
}
