// oz_gemm.cu -- FP64 matrix products emulated on the BF16 tensor cores
// (Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012).
//
//   C (M x N, FP64) = alpha op(A) op(B) + beta C
//
// GB300 runs FP64 at ~1.05 TFLOP/s and BF16 at ~1950 TFLOP/s.  Each row r of
// op(A) is written as 2^{eA_r} sum_{s=1..S} a_s 2^{-7s} with integer digits
// |a_s| <= 127 (exact in BF16), each column c of op(B) likewise; then
//   (op(A) op(B))(r,c) = 2^{eA_r + eB_c} sum_d 2^{-7d} sum_{s+t=d} (a_s b_t^T)(r,c).
// With S = 8 digits (56 bits) and the digit pairs s + t <= S + 1 kept, the
// truncation error is below 9.06 K 2^{-56} 2^{eA_r + eB_c} (the dropped pairs
// weigh 2^{-70} each), and the double-float fold adds at most
// 72 ceil(K / 128) 2^{-48} sum_k |a_k b_k|.  One tcgen05 accumulator per digit sum d
// lives in TMEM (8 x 32 FP32 columns per 128 x 32 output tile, two buffers);
// every 128 of K the partial sums are exact integers in FP32 (<= 8 pairs x
// 128 x 127^2 < 2^24), and they are folded into double-float (hi, lo) FP32
// registers with exact power-of-two weights.  The final value gets one FP64
// epilogue per element.
//
// Splitting works on the FP64 bit pattern with integer instructions only
// (GB300's FP64 pipe would make a floating-point split cost more than the
// product): significand m (53 bits), exponent E; the row scale eA_r is the
// largest E+1 of the row; the digits are the top 7S bits of m aligned to it.
// A split operand (OzOperand) can serve several products: its digit planes
// are addressed by a row offset, so a split of T(:, k0:n) by rows also
// serves products with the row block T(k0:m, k0:n).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr int OZ_S = 8;         // digits per operand
constexpr int OZ_TM = 128;      // output rows per CTA (UMMA M)
constexpr int OZ_TK = 64;       // K per stage (128 bytes of BF16)
constexpr int OZ_CHUNK = 2;     // k-blocks per exact FP32 chunk (K = 128)
constexpr long long kOzWait = 1LL << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
    const uint32_t a = su32(b);
    for (long long i = 0; i < kOzWait; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, uint64_t* b, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"((uint64_t)m), "r"(su32(b)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// ---------------------------------------------------------------- splitting
// Everything here is integer or FP32 work: on GB300 one FP64 instruction
// (even a compare) costs a warp 64 clocks of its SM sub-partition's FP64
// unit, and the int-to-float conversions run at a quarter of the ALU rate.
//
// Biased exponent field of a double: 0 for zero / subnormal, 2047 for
// Inf / NaN.
__device__ __forceinline__ int bexp_of(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

// row scale from the largest biased exponent of the row: |x| < 2^(be - 1022);
// rows of zeros / subnormals give INT_MIN so they never set a scale
__device__ __forceinline__ int scale_of(int maxbe) { return maxbe == 0 ? INT_MIN : maxbe - 1022; }

// row maxima of the exponent: L(r, k) = trans ? X(k, r) : X(r, k)
__global__ void k_oz_rowexp(const double* __restrict__ X, int64_t ld, int R, int K, bool trans, int* __restrict__ e,
                            int* status, DevGate gate) {
    if (gate_closed(gate)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (trans) {  // row r = column r of X: contiguous, one warp per row
        for (int r = blockIdx.x * 8 + warp; r < R; r += gridDim.x * 8) {
            int m = 0;
            for (int k = lane; k < K; k += 32) m = max(m, bexp_of(X[k + (int64_t)r * ld]));
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) {
                if (m == 0x7FF) atomicOr(status, ST_NONFINITE);
                e[r] = scale_of(m);
            }
        }
    } else {  // row r strided: 32 rows per block, lanes over rows, warps over k
        __shared__ int sm[8][33];
        const int r0 = blockIdx.x * 32;
        const int r = r0 + lane;
        int m = 0;
        if (r < R)
            for (int k = warp; k < K; k += 8) m = max(m, bexp_of(X[r + (int64_t)k * ld]));
        sm[warp][lane] = m;
        __syncthreads();
        if (warp == 0 && r < R) {
            int mm = sm[0][lane];
            for (int w = 1; w < 8; ++w) mm = max(mm, sm[w][lane]);
            if (mm == 0x7FF) atomicOr(status, ST_NONFINITE);
            e[r] = scale_of(mm);
        }
    }
}

// digits of x against the row scale er: F = floor(|x| 2^(7S - er)) < 2^56,
// digit s = bits 7(S-1-s) .. 7(S-1-s)+6 of F, signed like x.  BF16 of a
// magnitude a < 2^7 without a conversion instruction: the float with bits
// 0x4B000000 | a is 2^23 + a, and subtracting 2^23 leaves a exactly.
__device__ __forceinline__ void digits_of(double x, int er, uint32_t* dg) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((bits >> 52) & 0x7FF);
    unsigned long long F = 0ull;
    if (be != 0 && er != INT_MIN) {
        const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        // |x| / 2^er = mant 2^{be - 1075 - er}; F = floor(that 2^{7S})
        const int sh = be - 1075 - er + 7 * OZ_S;
        if (sh >= 0) F = mant << sh;  // F < 2^{7S} <= 2^56 since |x| < 2^er
        else if (sh > -64) F = mant >> (-sh);
    }
    const uint32_t sgn = (uint32_t)(bits >> 63) << 15;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        const uint32_t a = (uint32_t)(F >> (7 * (OZ_S - 1 - s))) & 127u;
        const float f = __int_as_float((int)(0x4B000000u | a)) - 8388608.0f;
        dg[s] = (__float_as_uint(f) >> 16) | sgn;
    }
}

// digits: Q[s][r][k] (s < OZ_S, row stride ldq, slice stride R*ldq) in BF16.
// trans: L(r, k) = X(k, r), four consecutive k per thread (one 8-byte store
// per digit plane); else a 32 x 32 tile is transposed through shared memory.
// Columns K..ldq-1 of Q are written as zeros, so that a product whose K is
// below one 64-wide k-block can read a whole block.
__global__ void k_oz_split(const double* __restrict__ X, int64_t ld, int R, int K, bool trans,
                           const int* __restrict__ e, uint16_t* __restrict__ Q, int64_t ldq, DevGate gate) {
    if (gate_closed(gate)) return;
    const size_t slice = (size_t)R * ldq;
    if (trans) {
        const int64_t kq = ldq / 4;
        const int64_t total = (int64_t)R * kq;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
            const int k = (int)(i % kq) * 4, r = (int)(i / kq);
            const int er = e[r];
            uint32_t dg[4][OZ_S];
#pragma unroll
            for (int u = 0; u < 4; ++u) digits_of(k + u < K ? X[k + u + (int64_t)r * ld] : 0.0, er, dg[u]);
            uint16_t* q = Q + (size_t)r * ldq + k;
#pragma unroll
            for (int s = 0; s < OZ_S; ++s)
                *reinterpret_cast<uint2*>(q + (size_t)s * slice) =
                    make_uint2(dg[0][s] | (dg[1][s] << 16), dg[2][s] | (dg[3][s] << 16));
        }
    } else {
        __shared__ double tile[32][33];
        const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
        for (int j = ty; j < 32; j += 8) {
            int r = r0 + tx, k = k0 + j;
            tile[j][tx] = (r < R && k < K) ? X[r + (int64_t)k * ld] : 0.0;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int r = r0 + j, k = k0 + tx;
            if (r < R && k < ldq) {
                uint32_t dg[OZ_S];
                digits_of(tile[tx][j], e[r], dg);
                uint16_t* q = Q + (size_t)r * ldq + k;
#pragma unroll
                for (int s = 0; s < OZ_S; ++s) q[(size_t)s * slice] = (uint16_t)dg[s];
            }
        }
    }
}

// ---------------------------------------------------------------- product
// Persistent kernel, one CTA per SM.  A job is one 128 x 32 output tile over
// one K range (a split-K slice).  CTAs take jobs from a global counter in
// order, so neighbouring column tiles run together and share the A digit
// tiles in L2, and a CTA that starts late (its SM busy with a concurrent
// kernel) simply takes fewer jobs.  The producer warp takes each job and
// passes its index to the MMA and drain warps through a 4-slot ring.
//   warp 8    : TMA producer (ring of OZ_AST stages of OZ_DPS A digit tiles,
//               ring of OZ_BST stacked B digit sets)
//   warp 9    : MMA issuer
//   warps 0-7 : drain TMEM into double-float registers, then the epilogue
// The 8 B digit planes of a k-block are stacked in shared memory (plane t =
// rows 32t .. 32t+31 of one 256-row operand), so all pairs (s, t), t <= 7-s,
// of A digit s are ONE MMA of N = 32 (8 - s) writing accumulator columns
// 32s .. 255, whose column block d then holds the digit sum d = s + t.  Two
// 256-column accumulator buffers alternate per 128-deep chunk: the drain of
// one chunk overlaps the MMAs of the next.  An A stage holds four digit
// tiles (two stages per k-block): each barrier round trip between the
// producer and MMA threads costs a few hundred cycles, as long as the MMAs
// of one digit tile, so fewer and larger stages keep the tensor pipe fed
// (a ten-stage ring of one tile each ran the split-K products 28%
// slower).
constexpr int OZ_TN = 32;                               // output columns per job
constexpr int OZ_DPS = 4;                               // A digit tiles per stage
constexpr int OZ_AST = 10 / OZ_DPS;                     // A ring stages
static_assert(OZ_S % OZ_DPS == 0, "whole digit tiles per stage");
constexpr int OZ_BST = 2;                               // B ring stages
constexpr int OZ_EPI = 8;                               // drain / epilogue warps
constexpr int OZ_THREADS = (OZ_EPI + 2) * 32;
constexpr int OZ_A_TILE = OZ_TM * OZ_TK * 2;            // 16 KB: one digit tile
constexpr int OZ_A_BYTES = OZ_DPS * OZ_A_TILE;          // one A stage
constexpr int OZ_BPLANE = OZ_TN * OZ_TK * 2;            // 4 KB
constexpr int OZ_B_BYTES = OZ_S * OZ_BPLANE;            // 32 KB
constexpr int OZ_ACC = OZ_S * OZ_TN;                    // 256 TMEM columns per buffer
// dynamic shared memory: the rings plus slack for the 1024-byte alignment
// (the barriers live in static shared memory)
constexpr int OZ_SMEM = OZ_AST * OZ_A_BYTES + OZ_BST * OZ_B_BYTES + 1024;

// FP32 value x times 2^sh, built as an FP64 bit pattern with integer
// instructions (exact); zero and FP32 subnormals give 0; returns false when
// the result would leave the FP64 normal range.
__device__ __forceinline__ bool f32_to_f64_scaled(float x, int sh, double& out) {
    const uint32_t u = __float_as_uint(x);
    const int e8 = (int)((u >> 23) & 0xFF);
    if (e8 == 0) { out = 0.0; return true; }
    const int e = e8 - 127 + 1023 + sh;
    if (e <= 0 || e >= 2047) return false;
    out = __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | ((unsigned long long)e << 52) |
                                           ((unsigned long long)(u & 0x7FFFFF) << 29)));
    return true;
}

struct OzJobs {
    int tiles_m, tiles_n, kbs, nkb_all, njobs;
    __device__ __forceinline__ void get(int j, int& m0, int& n0, int& z, int& kb0, int& nkb) const {
        const int tn = j % tiles_n, rest = j / tiles_n;
        m0 = (rest % tiles_m) * OZ_TM;
        n0 = tn * OZ_TN;
        z = rest / tiles_m;
        kb0 = z * kbs;
        nkb = min(nkb_all, kb0 + kbs) - kb0;
    }
};

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapB, int M, int N,
                                                            const int* __restrict__ eA, const int* __restrict__ eB,
                                                            double alpha, double beta, double* __restrict__ C,
                                                            int64_t ldc, OzJobs jb, double* __restrict__ P,
                                                            int* status, int a_plane, int a_row0, int b_plane,
                                                            int b_row0, int amode, int bmode, int* jobctr,
                                                            DevGate gate) {
    if (gate_closed(gate)) return;
    extern __shared__ __align__(1024) uint8_t oz_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* Abuf = sm;                                   // OZ_AST x OZ_A_BYTES
    uint8_t* Bbuf = sm + OZ_AST * OZ_A_BYTES;             // OZ_BST x 32 KB
    __shared__ __align__(8) uint64_t bars[2 * OZ_AST + 2 * OZ_BST + 2 + 2 + 4 + 4];
    __shared__ uint32_t tslot[1];
    uint64_t* a_full = bars;                   // [OZ_AST]
    uint64_t* a_empty = a_full + OZ_AST;       // [OZ_AST]
    uint64_t* b_full = a_empty + OZ_AST;       // [OZ_BST]
    uint64_t* b_empty = b_full + OZ_BST;       // [OZ_BST]
    uint64_t* acc_full = b_empty + OZ_BST;     // [2] chunk accumulated
    uint64_t* acc_empty = acc_full + 2;        // [2] chunk drained
    uint64_t* job_full = acc_empty + 2;        // [4] job index published
    uint64_t* job_empty = job_full + 4;        // [4] job index read by all
    __shared__ volatile int s_abort;
    __shared__ volatile int s_job[4];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool partial = jb.njobs > jb.tiles_m * jb.tiles_n;  // split-K: FP64 partials to P
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < OZ_AST; ++i) {
            bar_init(&a_full[i], 1);
            bar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < OZ_BST; ++i) {
            bar_init(&b_full[i], 1);
            bar_init(&b_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(&acc_full[i], 1);
            bar_init(&acc_empty[i], OZ_EPI);
        }
        for (int i = 0; i < 4; ++i) {
            bar_init(&job_full[i], 1);
            bar_init(&job_empty[i], 1 + OZ_EPI);  // the MMA warp and every drain warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(2u * OZ_ACC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == OZ_EPI) {
        if (lane == 0) {  // ---------------- TMA producer
            long long ia = 0, ib = 0;
            int jnext = atomicAdd(jobctr, 1);  // fetched one job ahead: the atomic's latency hides
            for (int n = 0; !s_abort; ++n) {   // behind the current job's copies
                const int slot = n & 3;
                if (!bar_wait(&job_empty[slot], (uint32_t)(((n >> 2) & 1) ^ 1))) { s_abort = 1; break; }
                const int j = jnext;
                if (j < jb.njobs) jnext = atomicAdd(jobctr, 1);
                s_job[slot] = (j < jb.njobs) ? j : -1;
                bar_arrive(&job_full[slot]);
                if (j >= jb.njobs) break;
                int m0, n0, z, kb0, nkb;
                jb.get(j, m0, n0, z, kb0, nkb);
                for (int kb = 0; kb < nkb && !s_abort; ++kb) {
                    const int k = (kb0 + kb) * OZ_TK;
                    const int sb = (int)(ib % OZ_BST);
                    if (!bar_wait(&b_empty[sb], (uint32_t)(((ib / OZ_BST) & 1) ^ 1))) { s_abort = 1; break; }
                    bar_expect(&b_full[sb], (uint32_t)OZ_B_BYTES);
                    for (int t = 0; t < OZ_S; ++t)
                        tma2d(Bbuf + sb * OZ_B_BYTES + t * OZ_BPLANE, &mapB, &b_full[sb], k, t * b_plane + b_row0 + n0);
                    ++ib;
                    for (int s0 = 0; s0 < OZ_S; s0 += OZ_DPS) {
                        const int sa = (int)(ia % OZ_AST);
                        if (!bar_wait(&a_empty[sa], (uint32_t)(((ia / OZ_AST) & 1) ^ 1))) { s_abort = 1; break; }
                        bar_expect(&a_full[sa], (uint32_t)OZ_A_BYTES);
                        for (int u = 0; u < OZ_DPS; ++u)
                            tma2d(Abuf + sa * OZ_A_BYTES + u * OZ_A_TILE, &mapA, &a_full[sa], k,
                                  (s0 + u) * a_plane + a_row0 + m0);
                        ++ia;
                    }
                }
            }
            // every copy issued must land before the CTA can exit
            for (long long i = (ib > OZ_BST ? ib - OZ_BST : 0); i < ib; ++i)
                bar_wait(&b_full[i % OZ_BST], (uint32_t)((i / OZ_BST) & 1));
            for (long long i = (ia > OZ_AST ? ia - OZ_AST : 0); i < ia; ++i)
                bar_wait(&a_full[i % OZ_AST], (uint32_t)((i / OZ_AST) & 1));
        }
    } else if (warp == OZ_EPI + 1) {
        if (lane == 0) {  // ---------------- MMA issuer
            long long ia = 0, ib = 0, chunk = 0;
            for (int n = 0; !s_abort; ++n) {
                const int slot = n & 3;
                if (!bar_wait(&job_full[slot], (uint32_t)((n >> 2) & 1))) { s_abort = 1; break; }
                const int j = s_job[slot];
                bar_arrive(&job_empty[slot]);
                if (j < 0) break;
                int m0, n0, z, kb0, nkb;
                jb.get(j, m0, n0, z, kb0, nkb);
                for (int kb = 0; kb < nkb && !s_abort; ++kb) {
                    const bool first = (kb % OZ_CHUNK) == 0;
                    const uint32_t buf = (uint32_t)(chunk & 1);
                    if (first) {
                        if (!bar_wait(&acc_empty[buf], (uint32_t)(((chunk >> 1) & 1) ^ 1))) { s_abort = 1; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    }
                    const int sb = (int)(ib % OZ_BST);
                    if (!bar_wait(&b_full[sb], (uint32_t)((ib / OZ_BST) & 1))) { s_abort = 1; break; }
                    const uint64_t db = desc_sw128(su32(Bbuf + sb * OZ_B_BYTES));
                    for (int s0 = 0; s0 < OZ_S; s0 += OZ_DPS) {
                        const int sa = (int)(ia % OZ_AST);
                        if (!bar_wait(&a_full[sa], (uint32_t)((ia / OZ_AST) & 1))) { s_abort = 1; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                        for (int u = 0; u < OZ_DPS; ++u) {
                            const int s = s0 + u;
                            const uint64_t da = desc_sw128(su32(Abuf + sa * OZ_A_BYTES + u * OZ_A_TILE));
                            const uint32_t dt = tmem + buf * OZ_ACC + (uint32_t)(s * OZ_TN);
                            // M = 128, N = 32 (8 - s), BF16 x BF16 -> FP32, both K-major
                            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                                   ((uint32_t)(((OZ_S - s) * OZ_TN) >> 3) << 17) |
                                                   ((uint32_t)(OZ_TM >> 4) << 24);
#pragma unroll
                            for (int k = 0; k < OZ_TK / 16; ++k) {
                                const uint64_t ko = (uint64_t)((k * 32) >> 4);
                                const uint32_t acc = (!first || s > 0 || k > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dt),
                                    "l"(da + ko), "l"(db + ko), "r"(idesc), "r"(acc)
                                    : "memory");
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         su32(&a_empty[sa]))
                                     : "memory");
                        ++ia;
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&b_empty[sb]))
                                 : "memory");
                    ++ib;
                    if ((kb % OZ_CHUNK) == OZ_CHUNK - 1 || kb == nkb - 1) {
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         su32(&acc_full[buf]))
                                     : "memory");
                        ++chunk;
                    }
                }
            }
        }
    } else {  // ---------------- warps 0-7: drain TMEM, epilogue
        const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32 quad.., columns 16 half..
        long long chunk = 0;
        for (int n = 0;; ++n) {
            const int slot = n & 3;
            const bool got = __all_sync(0xffffffffu, bar_wait(&job_full[slot], (uint32_t)((n >> 2) & 1)));
            if (!got || s_abort) {
                if (!got && lane == 0) atomicOr(status, ST_TIMEOUT);
                s_abort = 1;
                break;
            }
            const int j = s_job[slot];
            __syncwarp();
            if (lane == 0) bar_arrive(&job_empty[slot]);
            if (j < 0) break;
            int m0, n0, z, kb0, nkb;
            jb.get(j, m0, n0, z, kb0, nkb);
            // this job's C tile, row exponent and column exponents are loaded
            // before the accumulators are waited for, so their latency hides
            // behind the MMAs (the tile is read and written by this job only)
            const int r = m0 + quad * 32 + lane;
            const int cb = n0 + half * 16;
            const int ncols = (r < M) ? min(16, N - cb) : 0;
            const int er = (ncols > 0) ? eA[r] : INT_MIN;
            int ec[16];
            double cv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                ec[c] = (c < ncols) ? eB[cb + c] : INT_MIN;
                cv[c] = (!partial && bmode != 0 && c < ncols) ? C[r + (int64_t)(cb + c) * ldc] : 0.0;
            }
            float hi[16], lo[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0.0f;
            const int nch = (nkb + OZ_CHUNK - 1) / OZ_CHUNK;
            bool ok = true;
            for (int ch = 0; ch < nch; ++ch, ++chunk) {
                const uint32_t buf = (uint32_t)(chunk & 1);
                ok = __all_sync(0xffffffffu, bar_wait(&acc_full[buf], (uint32_t)((chunk >> 1) & 1)));
                if (!ok || s_abort) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + buf * OZ_ACC + (uint32_t)(half * 16);
#pragma unroll 1
                for (int g = 1; g >= 0; --g) {  // digit sums 7..4, then 3..0: four loads, one wait
                    uint32_t v[4][16];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint32_t ta = tbase + (uint32_t)((4 * g + 3 - i) * OZ_TN);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                            "%13,%14,%15}, [%16];"
                            : "=r"(v[i][0]), "=r"(v[i][1]), "=r"(v[i][2]), "=r"(v[i][3]), "=r"(v[i][4]),
                              "=r"(v[i][5]), "=r"(v[i][6]), "=r"(v[i][7]), "=r"(v[i][8]), "=r"(v[i][9]),
                              "=r"(v[i][10]), "=r"(v[i][11]), "=r"(v[i][12]), "=r"(v[i][13]), "=r"(v[i][14]),
                              "=r"(v[i][15])
                            : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int d = 4 * g + 3 - i;
                        const float w = __int_as_float((127 - 7 * (d + 2)) << 23);  // 2^{-7(d+2)}
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            float s, e;
                            two_sum(hi[c], __uint_as_float(v[i][c]) * w, s, e);
                            hi[c] = s;
                            lo[c] += e;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {  // renormalise (fast two-sum)
                    float s = hi[c] + lo[c];
                    lo[c] = lo[c] - (s - hi[c]);
                    hi[c] = s;
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) bar_arrive(&acc_empty[buf]);
            }
            if (!ok || s_abort) {
                if (!ok && lane == 0) atomicOr(status, ST_TIMEOUT);
                s_abort = 1;
                break;
            }
            if (ncols > 0) {
                // amode: 1 alpha = +1, 2 alpha = -1 (folded into the sign), 0 general
                const long long sgn = (amode == 2) ? (long long)(1ull << 63) : 0ll;
                double* Pz = partial ? P + (size_t)z * (size_t)M * (size_t)N : nullptr;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (c >= ncols) continue;
                    double v = 0.0;
                    if (er != INT_MIN && ec[c] != INT_MIN) {
                        double dh, dl;
                        if (amode != 0 && f32_to_f64_scaled(hi[c], er + ec[c], dh) &&
                            f32_to_f64_scaled(lo[c], er + ec[c], dl)) {
                            v = __longlong_as_double(__double_as_longlong(dh) ^ sgn) +
                                __longlong_as_double(__double_as_longlong(dl) ^ sgn);
                        } else {  // general alpha or extreme exponents
                            const double scale = ldexp(alpha, er + ec[c]);
                            v = fma((double)hi[c], scale, (double)lo[c] * scale);
                        }
                    }
                    if (partial) {
                        Pz[r + (size_t)(cb + c) * M] = v;
                    } else {
                        // bmode: 0 beta = 0, 1 beta = 1, 2 general
                        C[r + (int64_t)(cb + c) * ldc] = (bmode == 0) ? v : (bmode == 1 ? cv[c] + v : fma(beta, cv[c], v));
                    }
                }
            }
        }
    }
    if (s_abort && tid == 0) atomicOr(status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * OZ_ACC) : "memory");
}

// C = sum_z P[z] (fixed order) + beta C
__global__ void k_oz_reduce(int M, int N, int S, const double* __restrict__ P, double beta, int bzero,
                            double* __restrict__ C, int64_t ldc, DevGate gate) {
    if (gate_closed(gate)) return;
    const int64_t total = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += P[(size_t)z * total + e];
        double* c = C + (e % M) + (e / M) * ldc;
        *c = bzero ? s : fma(beta, *c, s);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool oz_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    auto enc = oz_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)OZ_TK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

unsigned oz_grid(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 8192)); }

}  // namespace

int64_t oz_ldq(int64_t K) { return (K + 63) / 64 * 64; }

// split-K factor: slices of whole 128-deep chunks until there are about
// eight jobs per SM (a shorter tail of the last wave); partials (FP64) need splits * M * N doubles
int oz_splits(int64_t M, int64_t N, int64_t K, int sms, size_t p_bytes) {
    const int64_t tiles = cdiv(M, OZ_TM) * cdiv(N, OZ_TN);
    const int64_t chunks = cdiv(cdiv(K, OZ_TK), OZ_CHUNK);
    int64_t s = 1;
    if (tiles < 8LL * sms) s = cdiv(8LL * sms, tiles);
    if (s > chunks) s = chunks;
    if (s > 64) s = 64;
    const int64_t fit = (int64_t)(p_bytes / (sizeof(double) * (size_t)M * (size_t)N));
    if (s > fit) s = fit;
    return (int)std::max<int64_t>(s, 1);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t oz_operand_bytes(int64_t R, int64_t K) {
    return align256(sizeof(uint16_t) * (size_t)OZ_S * (size_t)R * (size_t)oz_ldq(K)) + align256(sizeof(int) * (size_t)R);
}

size_t oz_work_bytes(int64_t M, int64_t N, int64_t K) {
    return oz_operand_bytes(M, K) + oz_operand_bytes(N, K) + 256 + sizeof(double) * ((size_t)1 << 27);
}

cudaError_t oz_split(bool trans, const double* X, int64_t ldx, int64_t R, int64_t K, void* buf, OzOperand* out,
                     int* status, cudaStream_t st) {
    const int64_t ldq = oz_ldq(K);
    uint16_t* Q = (uint16_t*)buf;
    int* e = (int*)((char*)buf + align256(sizeof(uint16_t) * (size_t)OZ_S * (size_t)R * (size_t)ldq));
    *out = OzOperand{Q, e, R, K, R, ldq};
    if (R <= 0 || K <= 0) return cudaSuccess;
    if (trans) {
        k_oz_rowexp<<<(unsigned)std::min<int64_t>(cdiv(R, 8), 4096), 256, 0, st>>>(X, ldx, (int)R, (int)K, true, e,
                                                                                      status, current_gate());
        k_oz_split<<<oz_grid(R * (ldq / 4)), 256, 0, st>>>(X, ldx, (int)R, (int)K, true, e, Q, ldq, current_gate());
    } else {
        k_oz_rowexp<<<(unsigned)cdiv(R, 32), 256, 0, st>>>(X, ldx, (int)R, (int)K, false, e, status, current_gate());
        k_oz_split<<<dim3((unsigned)cdiv(R, 32), (unsigned)cdiv(ldq, 32)), 256, 0, st>>>(X, ldx, (int)R, (int)K,
                                                                                          false, e, Q, ldq,
                                                                                          current_gate());
    }
    trace_count(2);
    return cudaGetLastError();
}

cudaError_t oz_product(const OzOperand& a, int64_t a_row0, const OzOperand& b, int64_t b_row0, int64_t M, int64_t N,
                       double alpha, double beta, double* C, int64_t ldc, double* P, size_t p_bytes, int sms,
                       int* status, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int64_t K = a.K;
    if (b.K != K || a_row0 < 0 || b_row0 < 0 || a_row0 + M > a.R || b_row0 + N > b.R) return cudaErrorInvalidValue;
    // a TMA box (128 or 32 rows) must fit inside the stacked digit planes; a
    // box that starts in plane s < 7 past the operand's rows reads the next
    // plane, and only feeds output rows / columns the epilogue discards
    if (OZ_S * a.plane < OZ_TM || OZ_S * b.plane < OZ_TN) return cudaErrorInvalidValue;
    // K below one k-block: the split wrote zeros up to ldq (>= 64), so the map
    // covers a whole block of them
    const int64_t kmap = K < OZ_TK ? a.ldq : K;
    if (K < OZ_TK && b.ldq != a.ldq) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!oz_map(&ma, a.Q, (int64_t)OZ_S * a.plane, kmap, a.ldq, OZ_TM)) return cudaErrorInvalidValue;
    if (!oz_map(&mb, b.Q, (int64_t)OZ_S * b.plane, kmap, b.ldq, OZ_TN)) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    OzJobs jb;
    jb.tiles_m = (int)cdiv(M, OZ_TM);
    jb.tiles_n = (int)cdiv(N, OZ_TN);
    jb.nkb_all = (int)cdiv(K, OZ_TK);
    const int s0 = oz_splits(M, N, K, sms, p_bytes > 256 ? p_bytes - 256 : 0);
    jb.kbs = (int)(cdiv(cdiv(jb.nkb_all, OZ_CHUNK), s0) * OZ_CHUNK);  // whole chunks per split
    const int splits = (int)cdiv(jb.nkb_all, jb.kbs);
    const int64_t njobs = (int64_t)jb.tiles_m * jb.tiles_n * splits;
    if (njobs > INT_MAX) return cudaErrorInvalidValue;
    jb.njobs = (int)njobs;
    const unsigned grid = (unsigned)std::min<int64_t>(njobs, sms);
    // the job counter sits in the first 256 bytes of P; the partials follow
    int* jobctr = (int*)P;
    P = (double*)((char*)P + 256);
    if (cudaMemsetAsync(jobctr, 0, sizeof(int), st) != cudaSuccess) return cudaErrorInvalidValue;
    const int amode = (alpha == 1.0) ? 1 : (alpha == -1.0 ? 2 : 0);
    const int bmode = (beta == 0.0) ? 0 : (beta == 1.0 ? 1 : 2);
    k_oz_gemm<<<grid, OZ_THREADS, OZ_SMEM, st>>>(ma, mb, (int)M, (int)N, a.e + a_row0, b.e + b_row0, alpha, beta, C,
                                                   ldc, jb, P, status, (int)a.plane, (int)a_row0, (int)b.plane,
                                                   (int)b_row0, amode, bmode, jobctr, current_gate());
    trace_count(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    k_oz_reduce<<<oz_grid(M * N), 256, 0, st>>>((int)M, (int)N, splits, P, beta, beta == 0.0 ? 1 : 0, C, ldc,
                                                  current_gate());
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t oz_gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work, size_t work_bytes,
                    int sms, int* status, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (M * OZ_S < OZ_TM || N * OZ_S < OZ_TN || K < 1) return cudaErrorInvalidValue;  // see oz_product
    // op(A) row r = column r of A when ta; op(B) column c = column c of B unless tb
    char* p = (char*)work;
    OzOperand a, b;
    cudaError_t e = oz_split(ta, A, lda, M, K, p, &a, status, st);
    if (e != cudaSuccess) return e;
    p += oz_operand_bytes(M, K);
    e = oz_split(!tb, B, ldb, N, K, p, &b, status, st);
    if (e != cudaSuccess) return e;
    p += oz_operand_bytes(N, K);
    double* P = (double*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    const size_t used = (size_t)((char*)P - (char*)work);
    return oz_product(a, 0, b, 0, M, N, alpha, beta, C, ldc, P, work_bytes > used ? work_bytes - used : 0, sms,
                      status, st);
}

}  // namespace rutv
