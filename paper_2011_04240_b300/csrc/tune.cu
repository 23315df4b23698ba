// Autotuner of the pair-kernel tiling.
//
// The pair step's tile has two free parameters that do not change any result
// (only which lanes and blocks do which pairs and samples): the lane group G
// (agents per group; a warp pairs groups of G agents, 32/G time samples per
// lane row) and QW, the number of consecutive time blocks a warp handles per
// work unit (larger units amortise the unit prologue and epilogue; smaller
// ones balance the persistent grid).  For float32 plans the apply mode is a
// third choice (one batched GEMM launch, or a matrix-vector product fused
// into the pair kernel), and so is the loop (the graph loop, or one block per
// instance running the whole loop).  amto_tune measures every candidate that fits on a
// synthetic batch of the caller's shape and reports them all.
//
// The best candidate is also kept in a process-wide cache keyed by the
// plan's shape (agents, samples, degree, batch rounded up to a power of two,
// precision, projection reading, multiplier form, obstacles, planar flag, rho
// stages, boundary rows); amto_create takes the cached choice for a plan of
// the same key whose tile, apply and loop are all automatic.  The cache can be
// written to and read from a text file.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "amto_internal.cuh"

namespace amto {
namespace {

// Deterministic synthetic start/goal sets: agents on a ring whose radius gives
// about 1.5 m between neighbours, goals on the opposite side and one metre
// higher; instance b rotates the ring by b radians.
void synthetic_inputs(int n, int batch, std::vector<float>& start, std::vector<float>& goal) {
    start.resize((size_t)batch * n * 3);
    goal.resize((size_t)batch * n * 3);
    const double r = std::fmax(2.0, 1.5 * n / (2.0 * M_PI));
    for (int b = 0; b < batch; ++b)
        for (int i = 0; i < n; ++i) {
            const double th = 2.0 * M_PI * i / n + b;
            float* s = &start[((size_t)b * n + i) * 3];
            float* g = &goal[((size_t)b * n + i) * 3];
            s[0] = (float)(r * std::cos(th));
            s[1] = (float)(r * std::sin(th));
            s[2] = 1.0f;
            g[0] = -s[0];
            g[1] = -s[1];
            g[2] = 2.0f;
        }
}

struct TuneKey {
    int n, m, degree, bucket, precision, proj_mode, multipliers, n_obs, planar, rho_stages;
    unsigned bc;
    bool operator==(const TuneKey& o) const {
        return n == o.n && m == o.m && degree == o.degree && bucket == o.bucket &&
               precision == o.precision && proj_mode == o.proj_mode &&
               multipliers == o.multipliers && n_obs == o.n_obs && planar == o.planar &&
               rho_stages == o.rho_stages && bc == o.bc;
    }
};

struct TuneChoice {
    TuneKey key;
    amto_tune_entry best;
};

std::mutex g_tune_mu;
std::vector<TuneChoice> g_tune;  // guarded by g_tune_mu

int batch_bucket(int b) {
    int k = 1;
    while (k < b) k <<= 1;
    return k;
}

TuneKey tune_key(const amto_params& p, int batch) {
    TuneKey k;
    k.n = p.n_agents;
    k.m = p.m_steps;
    k.degree = p.poly_degree;
    k.bucket = batch_bucket(batch);
    k.precision = p.precision;
    k.proj_mode = p.proj_mode;
    k.multipliers = p.multipliers;
    k.n_obs = p.n_obstacles;
    k.planar = p.planar;
    k.rho_stages = p.rho_stages > 1 ? p.rho_stages : 1;
    k.bc = p.bc_mask;
    return k;
}

void tune_put(const TuneKey& k, const amto_tune_entry& e) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (TuneChoice& c : g_tune)
        if (c.key == k) {
            c.best = e;
            return;
        }
    g_tune.push_back({k, e});
}

struct DeviceBuffers {
    float *start = nullptr, *goal = nullptr, *xi = nullptr, *resid = nullptr;
    int* iters = nullptr;
    ~DeviceBuffers() {
        cudaFree(start);
        cudaFree(goal);
        cudaFree(xi);
        cudaFree(resid);
        cudaFree(iters);
    }
};

}  // namespace

bool tune_lookup(const amto_params& p, amto_params* out) {
    if (p.tile_group != 0 || p.tile_time_blocks != 0 || p.apply_mode != AMTO_APPLY_AUTO ||
        p.loop_mode != AMTO_LOOP_AUTO)
        return false;
    const TuneKey k = tune_key(p, p.max_batch);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneChoice& c : g_tune)
        if (c.key == k) {
            *out = p;
            out->tile_group = c.best.tile_group;
            out->tile_time_blocks = c.best.tile_time_blocks;
            out->apply_mode = c.best.apply_mode;
            out->loop_mode = c.best.loop_mode;
            return true;
        }
    return false;
}

}  // namespace amto

using namespace amto;

extern "C" void amto_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

extern "C" int amto_tune_cache_size(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int)g_tune.size();
}

static const char kTuneMagic[] = "amto-tune-v1";

extern "C" amto_status amto_tune_cache_save(const char* path) {
    clear_error();
    if (!path) {
        set_error("invalid argument: path is NULL");
        return AMTO_EINVAL;
    }
    FILE* f = fopen(path, "w");
    if (!f) {
        set_error(std::string("cannot open ") + path + " for writing");
        return AMTO_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TuneChoice& c : g_tune) {
        const TuneKey& k = c.key;
        fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %u %d %d %d %d %.6f\n", kTuneMagic, k.n, k.m,
                k.degree, k.bucket, k.precision, k.proj_mode, k.multipliers, k.n_obs, k.planar,
                k.rho_stages, k.bc, c.best.tile_group, c.best.tile_time_blocks, c.best.apply_mode,
                c.best.loop_mode, c.best.us_per_iteration);
    }
    const bool ok = fclose(f) == 0;
    if (!ok) {
        set_error(std::string("writing ") + path + " failed");
        return AMTO_EINVAL;
    }
    return AMTO_OK;
}

extern "C" amto_status amto_tune_cache_load(const char* path) {
    clear_error();
    if (!path) {
        set_error("invalid argument: path is NULL");
        return AMTO_EINVAL;
    }
    FILE* f = fopen(path, "r");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return AMTO_EINVAL;
    }
    std::vector<TuneChoice> in;
    char line[512];
    int lineno = 0;
    amto_status st = AMTO_OK;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        if (line[0] == '\n' || line[0] == '#') continue;
        char magic[32] = {0};
        TuneChoice c{};
        TuneKey& k = c.key;
        const int got = sscanf(line, "%31s %d %d %d %d %d %d %d %d %d %d %u %d %d %d %d %lf", magic,
                               &k.n, &k.m, &k.degree, &k.bucket, &k.precision, &k.proj_mode,
                               &k.multipliers, &k.n_obs, &k.planar, &k.rho_stages, &k.bc,
                               &c.best.tile_group, &c.best.tile_time_blocks, &c.best.apply_mode,
                               &c.best.loop_mode, &c.best.us_per_iteration);
        const int G = c.best.tile_group, QW = c.best.tile_time_blocks;
        if (got != 17 || strcmp(magic, kTuneMagic) != 0 || !(G == 8 || G == 16 || G == 32) ||
            QW < 1 || QW > 8 || c.best.apply_mode < AMTO_APPLY_BATCHED ||
            c.best.apply_mode > AMTO_APPLY_FUSED || c.best.loop_mode < AMTO_LOOP_GRAPH ||
            c.best.loop_mode > AMTO_LOOP_BLOCK) {
            set_error(std::string(path) + ": line " + std::to_string(lineno) +
                      " is not a tuning entry");
            st = AMTO_EINVAL;
            break;
        }
        in.push_back(c);
    }
    fclose(f);
    if (st != AMTO_OK) return st;
    for (const TuneChoice& c : in) tune_put(c.key, c.best);
    return AMTO_OK;
}

extern "C" amto_status amto_tune(const amto_params* params, int batch, int iters,
                                 amto_tune_result* out) {
    clear_error();
    if (!params || !out) {
        set_error("invalid argument: params and out are required");
        return AMTO_EINVAL;
    }
    amto_params base = *params;
    base.tile_group = 0;
    base.tile_time_blocks = 0;
    base.apply_mode = AMTO_APPLY_AUTO;
    base.loop_mode = AMTO_LOOP_AUTO;
    if (validate_params(base) != AMTO_OK) return AMTO_EINVAL;
    if (batch < 1 || batch > base.max_batch || iters < 1 || iters > 100000) {
        set_error("invalid argument: 1 <= batch <= max_batch and 1 <= iters <= 100000");
        return AMTO_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    out->best = -1;
    const int n = base.n_agents, nv = base.poly_degree + 1;
    std::vector<float> hs, hg;
    synthetic_inputs(n, batch, hs, hg);
    DeviceBuffers d;
    const size_t in_b = sizeof(float) * hs.size();
    AMTO_CUDA_TRY(cudaMalloc((void**)&d.start, in_b));
    AMTO_CUDA_TRY(cudaMalloc((void**)&d.goal, in_b));
    AMTO_CUDA_TRY(cudaMalloc((void**)&d.xi, sizeof(float) * (size_t)batch * 3 * n * nv));
    AMTO_CUDA_TRY(cudaMalloc((void**)&d.resid, sizeof(float) * batch));
    AMTO_CUDA_TRY(cudaMalloc((void**)&d.iters, sizeof(int) * batch));
    AMTO_CUDA_TRY(cudaMemcpy(d.start, hs.data(), in_b, cudaMemcpyHostToDevice));
    AMTO_CUDA_TRY(cudaMemcpy(d.goal, hg.data(), in_b, cudaMemcpyHostToDevice));
    cudaStream_t s;
    AMTO_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    amto_status st = AMTO_OK;
    // loop time per iteration: difference of two solves (setup, initial
    // projection and the final residual cancel)
    auto timed = [&](amto_plan pl, int k, float* ms) -> amto_status {
        cudaEventRecord(e0, s);
        amto_status r = amto_solve(pl, batch, d.start, d.goal, nullptr, nullptr, nullptr, k, 0.f,
                                   d.xi, d.resid, d.iters, s);
        if (r != AMTO_OK) return r;
        cudaEventRecord(e1, s);
        AMTO_CUDA_TRY(cudaEventSynchronize(e1));
        AMTO_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        return AMTO_OK;
    };
    const int groups[3] = {8, 16, 32};
    const int qws[4] = {1, 2, 4, 8};
    // (apply mode, loop mode): batched + graph, fused + graph, batched + block
    const int modes[3] = {AMTO_APPLY_BATCHED, AMTO_APPLY_FUSED, AMTO_APPLY_BATCHED};
    const int loops[3] = {AMTO_LOOP_GRAPH, AMTO_LOOP_GRAPH, AMTO_LOOP_BLOCK};
    const int n_modes = base.precision == AMTO_PREC_FP32 ? 3 : 1;
    for (int mi = 0; mi < n_modes && st == AMTO_OK; ++mi)
    for (int gi = 0; gi < 3 && st == AMTO_OK; ++gi) {
        const int G = groups[gi];
        if (G > 8 && G / 2 >= n) continue;  // a group twice as wide as the instance
        for (int qi = 0; qi < 4 && st == AMTO_OK; ++qi) {
            amto_params p = base;
            p.tile_group = G;
            p.tile_time_blocks = qws[qi];
            p.apply_mode = modes[mi];
            p.loop_mode = loops[mi];
            p.max_batch = batch;
            if (loops[mi] == AMTO_LOOP_BLOCK && qws[qi] > 1) continue;  // no time blocks per warp
            const PairGeom g = choose_geometry(n, p.m_steps, G, qws[qi], batch, false);
            if (qws[qi] > 1 && g.TC / 2 >= p.m_steps) continue;  // one unit covers the horizon
            if (validate_params(p) != AMTO_OK) {
                clear_error();
                continue;
            }
            if (out->n_entries >= AMTO_TUNE_MAX) break;
            amto_plan pl = nullptr;
            st = amto_create(&p, &pl);
            if (st != AMTO_OK) break;
            float t_short = 0.f, t_long = 0.f, ms;
            st = timed(pl, 2, &ms);  // warm-up: graph instantiation
            if (st == AMTO_OK) st = timed(pl, 2, &t_short);
            if (st == AMTO_OK) st = timed(pl, 2 + iters, &t_long);
            amto_destroy(pl);
            if (st != AMTO_OK) break;
            amto_tune_entry& e = out->entries[out->n_entries];
            e.tile_group = G;
            e.tile_time_blocks = qws[qi];
            e.apply_mode = modes[mi];
            e.loop_mode = loops[mi];
            e.us_per_iteration = 1e3 * (double)(t_long - t_short) / iters;
            if (out->best < 0 || e.us_per_iteration < out->entries[out->best].us_per_iteration)
                out->best = out->n_entries;
            out->n_entries += 1;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (st == AMTO_OK && out->best < 0) {
        set_error("no tiling fits these parameters");
        st = AMTO_EINVAL;
    }
    if (st == AMTO_OK) tune_put(tune_key(base, batch), out->entries[out->best]);
    return st;
}
