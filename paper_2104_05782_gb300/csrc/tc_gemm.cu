// tc_gemm.cu -- BF16/FP16 x BF16/FP16 -> FP32 products on the tcgen05 tensor
// cores, for the low-precision sketch of Sec. 3.2.1 (Y = T22^T G and the power
// iteration Z = T22 Y, Y = T22^T Z).
//
//   C (M x N, FP32) = A (M x K) * B (N x K)^T,   A and B K-major (row-major with
//   K contiguous), N <= 256 (N = the block size b, one tile), K split over
//   gridDim.y slices (deterministic partials, reduced by the caller).
//
// At b = 128 the product does b flops per byte of A read, far below the
// BF16 ridge of GB300 (~280 flop/B), so the kernel is HBM bound: what matters
// is streaming A at full bandwidth.  Design: one 128-row output tile per CTA,
// a TMA producer thread (cp.async.bulk.tensor, 128B swizzle) filling a ring
// of 4-6 shared-memory stages, one thread issuing tcgen05.mma (M=128, N=b,
// K=16) into a TMEM accumulator of N FP32 columns, stages released by
// tcgen05.commit, and four warps draining TMEM with tcgen05.ld (32x32b) into
// coalesced column-major FP32 stores.  Every mbarrier wait is bounded; a wait
// that runs out records ST_TIMEOUT, drains what is in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr int TM = 128;       // rows per tile (UMMA M)
constexpr int TK = 64;        // K elements per stage (128 bytes of 16-bit values)
constexpr int UK = 16;        // K per tcgen05.mma (kind::f16)
constexpr int NTHR = 128;
constexpr long long kWaitLimit = 1LL << 24;
constexpr int kMaxSplits = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row (1024-byte) swizzle atoms.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                            // descriptor version (sm_100 family)
    d |= (uint64_t)2 << 61;                            // swizzle mode: 128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = BF16 (1) or F16 (0), both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, int ab_fmt) {
    return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int N, int STAGES>
struct SmemLayout {
    static constexpr int A_BYTES = TM * TK * 2;
    static constexpr int B_BYTES = N * TK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TOTAL = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
};

template <int N, int STAGES>
__global__ void __launch_bounds__(NTHR, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB, int M, int K,
                                                      int kblocks_per_split, uint32_t idesc, float* __restrict__ C,
                                                      int64_t ldc, int64_t split_stride, int* status, DevGate gate) {
    if (gate_closed(gate)) return;
    using L = SmemLayout<N, STAGES>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * L::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TM;
    const int nkb_total = (K + TK - 1) / TK;
    const int kb0 = blockIdx.y * kblocks_per_split;
    const int kb1 = min(nkb_total, kb0 + kblocks_per_split);
    const int nkb = max(0, kb1 - kb0);
    float* Cz = C + (size_t)blockIdx.y * (size_t)split_stride;

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (nkb > 0) {
        if (warp == 0 && lane == 0) {
            // TMA producer
            int issued = 0;
            for (int it = 0; it < nkb; ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&empty[s], ph ^ 1u) || s_abort) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                uint8_t* sa = smem + s * L::STAGE;
                uint8_t* sb = sa + L::A_BYTES;
                mbar_expect_tx(&full[s], (uint32_t)L::STAGE);
                const int kx = (kb0 + it) * TK;
                tma_load_2d(sa, &mapA, &full[s], kx, m0);
                tma_load_2d(sb, &mapB, &full[s], kx, 0);
                issued = it + 1;
            }
            // drain: every issued stage must have landed before the CTA exits
            for (int it = max(0, issued - STAGES); it < issued; ++it)
                mbar_wait(&full[it % STAGES], (uint32_t)((it / STAGES) & 1));
        } else if (warp == 1 && lane == 0) {
            // MMA issuer
            int committed = 0;
            for (int it = 0; it < nkb; ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&full[s], ph) || s_abort) {
                    atomicOr(status, ST_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(smem + s * L::STAGE);
                const uint32_t sb = sa + L::A_BYTES;
                const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
                for (int k = 0; k < TK / UK; ++k) {
                    const uint64_t koff = (uint64_t)((k * UK * 2) >> 4);
                    const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(da + koff), "l"(db + koff), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
                committed = it + 1;
            }
            (void)committed;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(done))
                         : "memory");
        }
        __syncwarp();
        // epilogue: all four warps wait for the accumulator
        const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0));
        if (!ok && lane == 0) atomicOr(status, ST_TIMEOUT);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        if (ok && !s_abort) {
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                      "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                      "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) Cz[row + (int64_t)(c0 + j) * ldc] = __uint_as_float(r[j]);
                }
            }
        }
    } else {
        // empty K slice: its partial is zero
        const int row = m0 + tid;
        if (row < M)
            for (int c = 0; c < N; ++c) Cz[row + (int64_t)c * ldc] = 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)N) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D tensor map of a row-major rows x cols 16-bit matrix (row stride ld
// elements), box = box_cols x box_rows, 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
              int box_cols, bool f16) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int N, int STAGES>
cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, int M, int K, int kbs, int splits,
                      uint32_t idesc, float* C, int64_t ldc, int64_t split_stride, int* status, cudaStream_t st) {
    using L = SmemLayout<N, STAGES>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<N, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::TOTAL);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((unsigned)cdiv(M, TM), (unsigned)splits);
    k_tc_gemm<N, STAGES><<<grid, NTHR, L::TOTAL, st>>>(ma, mb, M, K, kbs, idesc, C, ldc, split_stride, status,
                                                       current_gate());
    trace_count(1);
    return cudaGetLastError();
}

}  // namespace

int tc_gemm_npad(int Nb) { return Nb <= 32 ? 32 : Nb <= 64 ? 64 : Nb <= 128 ? 128 : 256; }

int tc_gemm_splits(int64_t M, int64_t K, int sms) {
    int64_t tiles = cdiv(M, TM);
    int64_t nkb = cdiv(K, TK);
    int64_t s = cdiv(sms, std::max<int64_t>(tiles, 1));
    if (s > nkb) s = nkb;
    if (s > kMaxSplits) s = kMaxSplits;
    if (s < 1) s = 1;
    return (int)s;
}

// C_z (M x Npad FP32, column-major, ldc) for z < splits = partial products of
// A (M x K, row stride lda) and B (Npad x K, row stride ldb), both 16-bit
// K-major; Npad = tc_gemm_npad(Nb) and the caller keeps rows Nb..Npad-1 of B
// zero.  Needs M >= 128, K >= 64, 16-byte aligned bases and ld % 8 == 0
// (TMA rules); otherwise returns cudaErrorInvalidValue without launching.
cudaError_t tc_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int Nb, int64_t K, bool f16,
                    float* C, int64_t ldc, int64_t split_stride, int splits, int* status, cudaStream_t st) {
    if (M <= 0 || Nb <= 0) return cudaSuccess;
    if (Nb > 256 || (lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
        return cudaErrorInvalidValue;
    const int N = tc_gemm_npad(Nb);
    if (M < TM || K < TK) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, TM, TK, f16)) return cudaErrorInvalidValue;
    if (!make_map(&mb, B, N, K, ldb, N, TK, f16)) return cudaErrorInvalidValue;
    const int fmt = f16 ? 0 : 1;
    int64_t nkb = cdiv(K, TK);
    int kbs = (int)cdiv(nkb, splits);
    switch (N) {
        case 32: return launch_tc<32, 6>(ma, mb, (int)M, (int)K, kbs, splits, make_idesc(TM, 32, fmt), C, ldc, split_stride, status, st);
        case 64: return launch_tc<64, 6>(ma, mb, (int)M, (int)K, kbs, splits, make_idesc(TM, 64, fmt), C, ldc, split_stride, status, st);
        case 128: return launch_tc<128, 6>(ma, mb, (int)M, (int)K, kbs, splits, make_idesc(TM, 128, fmt), C, ldc, split_stride, status, st);
        default: return launch_tc<256, 4>(ma, mb, (int)M, (int)K, kbs, splits, make_idesc(TM, 256, fmt), C, ldc, split_stride, status, st);
    }
}

}  // namespace rutv
