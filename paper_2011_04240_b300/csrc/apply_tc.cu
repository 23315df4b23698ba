// Batched cached-inverse apply on the 5th-generation tensor cores (sm_103a):
//   xi[col][row] += sum_k K^-1_top[row][k] * rhs[col][k]
// for all same-n instances of a batch at once (Eq. kkt_step_x, Remark 1: the
// inverse is shared, so the batch turns the per-instance GEMV into one GEMM
// of (n nv) x 3B x kdim).
//
// One block computes a 128 x 128 output tile over a slice of K:
//   warp 0 lane 0   TMA producer: 2-D tiled bulk-tensor loads (128-byte
//                   swizzle) of the K^-1 tile and the right-hand-side tile,
//                   each split into a "hi" part (TF32, or BF16) and the
//                   residual "lo" part (float32, or BF16), into a 3-stage
//                   shared-memory ring;
//   warp 1 lane 0   MMA issuer: tcgen05.mma kind::tf32 (K = 8 per MMA) or
//                   kind::f16 with BF16 operands (K = 16 per MMA; both are
//                   32 bytes of a 128-byte swizzled row), accumulator in
//                   tensor memory (128 lanes x 128 float32 columns), three
//                   products per k-step (hi*hi + hi*lo + lo*hi, the split
//                   ("x3") correction), or one (plain TF32 / BF16);
//   all 4 warps     epilogue: tcgen05.ld of the accumulator, then either an
//                   add into xi or a split-K partial (summed in split order
//                   by the separate reduce kernel).
// All mbarrier waits are bounded; on timeout the block records an error in
// the solve's control block, drains what it issued (bounded) and frees its
// tensor memory.
#include <cuda.h>

#include <cstdint>

#include "amto_internal.cuh"

namespace amto {
namespace {

constexpr int kBM = 128, kBN = 128, kTcStages = 3;
constexpr int kRowBytes = 128;                       // one swizzled K row of a tile
constexpr int kTileBytes = kBM * kRowBytes;          // 16 KB (kBN == kBM)
constexpr int kTcStageBytes = 4 * kTileBytes;       // A hi, A lo, B hi, B lo
constexpr unsigned kTcPolls = 1u << 22;

__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned parity) {
    for (unsigned i = 0; i < kTcPolls; ++i)
        if (tc_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tc_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major operand tile written by TMA with
// 128-byte swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}
// Instruction descriptors: D float32, A and B both K-major, N x M tile;
// operand format TF32 (kind::tf32) or BF16 (kind::f16).
constexpr uint32_t kIdescShape = ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | kIdescShape;
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | kIdescShape;

template <bool BF>
__device__ __forceinline__ void mma_step(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    if (BF)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(kIdescBf16), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
            : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 columns of the 32 lanes a warp owns, one 32-bit value each.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
        "%26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
          "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
          "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
          "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

struct TcArgs {
    int M, K, N, kper, splits, x3;
    int adapt;          // per-instance switch: correction products in a second accumulator
    const int* px3;     // [B] instances that have switched (adapt)
    float* xi;          // [N][M]
    const int* flags;
    float* ws;          // [splits][N][M]
    Ctl* ctl;
};

// Tensor maps of the K^-1 operands of every rho stage and of the right-hand
// sides (kernel parameters: the descriptors must live in parameter space).
struct TcMaps {
    CUtensorMap a_hi[kMaxRhoStages];
    CUtensorMap a_lo[kMaxRhoStages];
    CUtensorMap b_hi, b_lo;
};

template <bool BF>
__global__ void __launch_bounds__(128, 1)
    k_apply_tc(const __grid_constant__ TcMaps TM, TcArgs A) {
    extern __shared__ unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long bars[2 * kTcStages + 1];
    __shared__ unsigned tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN, kz = blockIdx.z;
    constexpr int kBK = BF ? kRowBytes / 2 : kRowBytes / 4;  // K elements per k-block
    const int kbeg = kz * A.kper, kend = min(A.K, kbeg + A.kper);
    const int nk = (kend - kbeg + kBK - 1) / kBK;
    const unsigned base = (su32(tc_smem) + 1023u) & ~1023u;  // 1024-byte aligned tiles
    const unsigned full0 = su32(&bars[0]), empty0 = su32(&bars[kTcStages]),
                   done = su32(&bars[2 * kTcStages]);
    const bool two_acc = A.adapt != 0;  // main and correction accumulators
    const uint32_t tcols = two_acc ? 2 * kBN : kBN;
    // tensor memory and barriers do not depend on the previous kernel: set
    // them up while it drains (programmatic dependent launch)
    if (warp == 0) {  // tensor memory for the 128 x 128 float32 accumulator(s)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kTcStages; ++s) {
            tc_mbar_init(full0 + 8 * s, 1);
            tc_mbar_init(empty0 + 8 * s, 1);
        }
        tc_mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    griddep_wait();
    const int stage = A.ctl->stage;  // rho stage of this QP solve (the batch is in step)
    const CUtensorMap& ta_hi = TM.a_hi[stage];
    const CUtensorMap& ta_lo = TM.a_lo[stage];
    const CUtensorMap& tb_hi = TM.b_hi;
    const CUtensorMap& tb_lo = TM.b_lo;
    unsigned* err = &A.ctl->error;
    // switch mode: the tile needs the correction products when any of its
    // columns' instances has switched (uniform over the block)
    bool corr = A.x3 != 0;
    if (A.adapt) {
        const int col = n0 + tid;  // kBN == blockDim.x
        corr = __syncthreads_or(col < A.N && A.px3[col / 3] != 0) != 0;
    }
    const uint32_t tmem = tmem_slot;
    const uint32_t tmem_c = two_acc ? tmem + (uint32_t)kBN : tmem;  // correction accumulator
    const unsigned tx_bytes = (unsigned)((corr ? 4 : 2) * kTileBytes);
    bool ok = true;

    if (tid == 0) {  // producer
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % kTcStages;
            if (kb >= kTcStages && !tc_wait(empty0 + 8 * s, ((kb / kTcStages) - 1) & 1)) {
                ok = false;
                atomicOr(err, 1u);
                break;
            }
            const unsigned st = base + s * kTcStageBytes, fb = full0 + 8 * s;
            const int kx = kbeg + kb * kBK;
            tc_expect_tx(fb, tx_bytes);
            tma_load_2d(st, &ta_hi, kx, m0, fb);
            tma_load_2d(st + 2 * kTileBytes, &tb_hi, kx, n0, fb);
            if (corr) {
                tma_load_2d(st + kTileBytes, &ta_lo, kx, m0, fb);
                tma_load_2d(st + 3 * kTileBytes, &tb_lo, kx, n0, fb);
            }
        }
    } else if (tid == 32) {  // MMA issuer
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % kTcStages;
            if (!tc_wait(full0 + 8 * s, (kb / kTcStages) & 1)) {
                ok = false;
                atomicOr(err, 1u);
                break;
            }
            tc_fence_after();
            const unsigned st = base + s * kTcStageBytes;
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk) {  // 32 bytes of K per MMA
                const uint64_t ah = smem_desc(st + kk * 32);
                const uint64_t bh = smem_desc(st + 2 * kTileBytes + kk * 32);
                mma_step<BF>(tmem, ah, bh, (kb > 0 || kk > 0) ? 1u : 0u);
                if (corr) {
                    const uint64_t al = smem_desc(st + kTileBytes + kk * 32);
                    const uint64_t bl = smem_desc(st + 3 * kTileBytes + kk * 32);
                    // x3: into the one accumulator; switch: into the second
                    mma_step<BF>(tmem_c, ah, bl, (two_acc && kb == 0 && kk == 0) ? 0u : 1u);
                    mma_step<BF>(tmem_c, al, bh, 1u);
                }
            }
            mma_commit(empty0 + 8 * s);  // the stage is free once these MMAs are done
        }
        mma_commit(done);
    }
    __syncwarp();
    // epilogue: wait for the accumulator (bounded), read it lane = row
    const bool have = __all_sync(0xffffffffu, tc_wait(done, 0));  // warp-uniform for tcgen05.ld
    if (!have && lane == 0) atomicOr(err, 1u);
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    const int N = A.N, M = A.M;
    if (have) {
        float* dst = (A.splits == 1) ? nullptr : A.ws + (size_t)kz * N * M;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
                "%26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                  "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                  "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (two_acc && corr) {  // switched columns add the correction accumulator
                uint32_t w[32];
                tmem_ld32(tmem_c + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, w);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N && A.px3[col / 3])
                        v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(w[j]));
                }
            }
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= N) continue;
                    const float val = __uint_as_float(v[j]);
                    if (dst) {
                        dst[(size_t)col * M + row] = val;
                    } else if (A.flags[col / 3] & FLAG_APPLY) {
                        A.xi[(size_t)col * M + row] += val;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols)
                     : "memory");
    // split-K partials are summed in split order by k_splitk_reduce
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Row-major matrix [rows][ld] of float32 (or BF16) with `cols` valid columns:
// 128-byte x 128-row boxes, 128-byte swizzle, zero fill outside.
amto_status make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, bool bf16) {
    const int es = bf16 ? 2 : 4;
    EncodeTiled enc = encoder();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return AMTO_ECUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)kBM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     2, const_cast<void*>(base), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return AMTO_ECUDA;
    }
    return AMTO_OK;
}
}  // namespace

size_t tc_smem_bytes() { return (size_t)kTcStages * kTcStageBytes + 1024; }

amto_status tc_configure(amto_plan_s* pl) {
    AMTO_CUDA_TRY(cudaFuncSetAttribute((void*)k_apply_tc<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes()));
    AMTO_CUDA_TRY(cudaFuncSetAttribute((void*)k_apply_tc<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes()));
    const int M = pl->n * pl->nv, K = pl->kdim, rows_b = 3 * pl->prm.max_batch;
    amto_status st = AMTO_OK;
    const bool bf = prec_bf16(pl->prm.precision);
    for (int j = 0; j < pl->sched.J && st == AMTO_OK; ++j) {
        if (bf) {
            st = make_map(&pl->tm_a_hi[j], pl->Kb_hi + j * pl->ks_bf, M, K, pl->kp8, true);
            if (st == AMTO_OK)
                st = make_map(&pl->tm_a_lo[j], pl->Kb_lo + j * pl->ks_bf, M, K, pl->kp8, true);
        } else {
            st = make_map(&pl->tm_a_hi[j], pl->Kt_hi + j * pl->ks_tc, M, K, pl->kp, false);
            if (st == AMTO_OK)
                st = make_map(&pl->tm_a_lo[j], pl->Kt_lo + j * pl->ks_tc, M, K, pl->kp, false);
        }
    }
    if (st == AMTO_OK)
        st = bf ? make_map(&pl->tm_b_hi, pl->rb_hi, rows_b, K, pl->kp8, true)
                : make_map(&pl->tm_b_hi, pl->rhs, rows_b, K, pl->kp, false);
    if (st == AMTO_OK)
        st = bf ? make_map(&pl->tm_b_lo, pl->rb_lo, rows_b, K, pl->kp8, true)
                : make_map(&pl->tm_b_lo, pl->rhs_lo, rows_b, K, pl->kp, false);
    return st;
}

void tc_shape(const amto_plan_s* pl, int batch, int* tm, int* tn, int* splits, int* kper) {
    const int M = pl->n * pl->nv, N = 3 * batch, K = pl->kdim;
    const int kbk = prec_bf16(pl->prm.precision) ? kRowBytes / 2 : kRowBytes / 4;
    *tm = (M + kBM - 1) / kBM;
    *tn = (N + kBN - 1) / kBN;
    // the split over K is fixed by the plan's reference batch, so a column's
    // summation order (hence its result) does not depend on the batch size
    const int tn_max = (3 * pl->ref_batch + kBN - 1) / kBN;
    int sp = pl->num_sms / (*tm * tn_max);  // one wave of one-block-per-SM tiles
    sp = sp < 1 ? 1 : (sp > 8 ? 8 : sp);
    int kp = (K + sp - 1) / sp;
    kp = (kp + kbk - 1) / kbk * kbk;
    *splits = (K + kp - 1) / kp;
    *kper = kp;
}

amto_status launch_apply_tc(amto_plan_s* pl, int batch, cudaStream_t s) {
    TcArgs a{};
    a.M = pl->n * pl->nv;
    a.K = pl->kdim;
    a.N = 3 * batch;
    a.x3 = pl->prm.precision == AMTO_PREC_TF32X3 || pl->prm.precision == AMTO_PREC_BF16X3;
    a.adapt = prec_adapt(pl->prm.precision) ? 1 : 0;
    a.px3 = pl->px3;
    a.xi = pl->xi;
    a.flags = pl->flags;
    a.ws = pl->gemm_ws;
    a.ctl = pl->ctl;
    int tm_, tn, sp;
    tc_shape(pl, batch, &tm_, &tn, &sp, &a.kper);
    a.splits = sp;
    static_assert(sizeof(TcMaps) + sizeof(TcArgs) < 32000, "kernel parameter space");
    TcMaps tm;
    for (int j = 0; j < kMaxRhoStages; ++j) {
        tm.a_hi[j] = pl->tm_a_hi[j < pl->sched.J ? j : 0];
        tm.a_lo[j] = pl->tm_a_lo[j < pl->sched.J ? j : 0];
    }
    tm.b_hi = pl->tm_b_hi;
    tm.b_lo = pl->tm_b_lo;
    if (prec_bf16(pl->prm.precision))
        AMTO_CUDA_TRY(launch_pdl(k_apply_tc<true>, dim3(tm_, tn, sp), dim3(128), tc_smem_bytes(),
                                 s, tm, a));
    else
        AMTO_CUDA_TRY(launch_pdl(k_apply_tc<false>, dim3(tm_, tn, sp), dim3(128), tc_smem_bytes(),
                                 s, tm, a));
    AMTO_CUDA_TRY(cudaGetLastError());
    if (sp > 1) return launch_splitk_reduce(pl, batch, sp, s);
    return AMTO_OK;
}

}  // namespace amto
