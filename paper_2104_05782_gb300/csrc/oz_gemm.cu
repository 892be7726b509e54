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
// error is about K 2^{-56} max|op(A)(r,:)| max|op(B)(:,c)| (digit truncation;
// the dropped pairs weigh 2^{-70}).  One tcgen05 accumulator per digit sum d
// lives in TMEM (8 x TN FP32 columns: all 512 for TN = 64, 256 for the
// TN = 32 tiles of short-K products, two CTAs per SM); every 128 of K the partial
// sums are exact integers in FP32 (<= 8 pairs x 128 x 127^2 < 2^24), and they
// are folded into double-float (hi, lo) FP32 registers with exact
// power-of-two weights.  The final value gets one FP64 epilogue per element.
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
constexpr int OZ_TN = 64;       // output columns per CTA (UMMA N); 32 for short-K products
constexpr int OZ_TK = 64;       // K per stage (128 bytes of BF16)
constexpr int OZ_CHUNK = 2;     // k-blocks per exact FP32 chunk (K = 128)
constexpr int OZ_THREADS = 192; // warps 0-3 drain TMEM, warp 4 = TMA, warp 5 = MMA
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
// Exponent E+1 of a nonzero finite double (|x| < 2^{E+1}); 0-exponent values
// (zero, subnormal) give INT_MIN so they never set the row scale.
__device__ __forceinline__ int exp_of(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((bits >> 52) & 0x7FF);
    return be == 0 ? INT_MIN : be - 1022;
}

// row maxima of the exponent: L(r, k) = trans ? X(k, r) : X(r, k)
__global__ void k_oz_rowexp(const double* __restrict__ X, int64_t ld, int R, int K, bool trans, int* __restrict__ e,
                            int* status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (trans) {  // row r = column r of X: contiguous, one warp per row
        for (int r = blockIdx.x * 8 + warp; r < R; r += gridDim.x * 8) {
            int m = INT_MIN;
            bool bad = false;
            for (int k = lane; k < K; k += 32) {
                double v = X[k + (int64_t)r * ld];
                bad |= !isfinite(v);
                m = max(m, exp_of(v));
            }
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
            if (lane == 0) e[r] = m;
        }
    } else {  // row r strided: 32 rows per block, lanes over rows, warps over k
        __shared__ int sm[8][33];
        const int r0 = blockIdx.x * 32;
        const int r = r0 + lane;
        int m = INT_MIN;
        bool bad = false;
        if (r < R)
            for (int k = warp; k < K; k += 8) {
                double v = X[r + (int64_t)k * ld];
                bad |= !isfinite(v);
                m = max(m, exp_of(v));
            }
        if (bad) atomicOr(status, ST_NONFINITE);
        sm[warp][lane] = m;
        __syncthreads();
        if (warp == 0 && r < R) {
            int mm = sm[0][lane];
            for (int w = 1; w < 8; ++w) mm = max(mm, sm[w][lane]);
            e[r] = mm;
        }
    }
}

// digits: Q[s][r][k] (s < OZ_S, row stride ldq, slice stride R*ldq) in BF16
__device__ __forceinline__ void split_one(double x, int er, uint16_t* out, size_t slice_stride) {
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
    const bool neg = (bits >> 63) != 0;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        int digit = (int)((F >> (7 * (OZ_S - 1 - s))) & 127ull);
        float f = (float)(neg ? -digit : digit);
        __nv_bfloat16 h = __float2bfloat16_rn(f);
        out[(size_t)s * slice_stride] = *reinterpret_cast<uint16_t*>(&h);
    }
}

__global__ void k_oz_split(const double* __restrict__ X, int64_t ld, int R, int K, bool trans,
                           const int* __restrict__ e, uint16_t* __restrict__ Q, int64_t ldq) {
    const size_t slice = (size_t)R * ldq;
    if (trans) {  // L(r, k) = X(k, r): k contiguous in memory and in Q
        const int64_t total = (int64_t)R * K;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
            const int k = (int)(i % K), r = (int)(i / K);
            split_one(X[k + (int64_t)r * ld], e[r], Q + (size_t)r * ldq + k, slice);
        }
    } else {  // L(r, k) = X(r, k): transpose through a 32 x 32 tile
        __shared__ double tile[32][33];
        const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
        const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
        for (int j = ty; j < 32; j += 8) {
            int r = r0 + tx, k = k0 + j;
            tile[j][tx] = (r < R && k < K) ? X[r + (int64_t)k * ld] : 0.0;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            int r = r0 + j, k = k0 + tx;
            if (r < R && k < K) split_one(tile[tx][j], e[r], Q + (size_t)r * ldq + k, slice);
        }
    }
}

// ---------------------------------------------------------------- product
template <int TN>
struct OzSmem {
    static constexpr int A_BYTES = OZ_TM * OZ_TK * 2;           // 16 KB
    static constexpr int B_BYTES = TN * OZ_TK * 2;              // 8 KB (TN = 64)
    static constexpr int B_SET = OZ_S * B_BYTES;                // 64 KB (TN = 64)
    static constexpr int TOTAL = 2 * A_BYTES + 2 * B_SET + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = OZ_S * TN;            // 512 or 256
};

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

template <int TN, int MINB>
__global__ void __launch_bounds__(OZ_THREADS, MINB) k_oz_gemm(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB, int M, int N,
                                                           int K, const int* __restrict__ eA,
                                                           const int* __restrict__ eB, double alpha, double beta,
                                                           double* __restrict__ C, int64_t ldc, int kbs,
                                                           double* __restrict__ P, int* status, int a_plane,
                                                           int a_row0, int b_plane, int b_row0) {
    using L = OzSmem<TN>;
    extern __shared__ __align__(1024) uint8_t oz_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* Abuf = sm;                               // 2 x A_BYTES
    uint8_t* Bbuf = sm + 2 * L::A_BYTES;              // 2 x B_SET
    uint64_t* bars = (uint64_t*)(sm + 2 * L::A_BYTES + 2 * L::B_SET);
    uint64_t* a_full = bars;       // [2]
    uint64_t* a_empty = bars + 2;  // [2]
    uint64_t* b_full = bars + 4;   // [2]
    uint64_t* b_empty = bars + 6;  // [2]
    uint64_t* c_full = bars + 8;   // chunk accumulated
    uint64_t* c_free = bars + 9;   // chunk drained
    uint32_t* tslot = (uint32_t*)(bars + 10);
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * OZ_TM, n0 = blockIdx.y * TN;
    // split z covers k-blocks [kb0, kb0 + nkb); gridDim.z > 1 writes FP64 partials to P
    const int nkb_all = (K + OZ_TK - 1) / OZ_TK;
    const int kb0 = blockIdx.z * kbs;
    const int nkb = max(0, min(nkb_all, kb0 + kbs) - kb0);
    const int nchunks = (nkb + OZ_CHUNK - 1) / OZ_CHUNK;
    const bool partial = gridDim.z > 1;

    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < 2; ++i) {
            bar_init(&a_full[i], 1);
            bar_init(&a_empty[i], 1);
            bar_init(&b_full[i], 1);
            bar_init(&b_empty[i], 1);
        }
        bar_init(c_full, 1);
        bar_init(c_free, 128);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 4) {
        if (lane == 0 && nkb > 0) {  // ---------------- TMA producer
            int ia = 0, kb_done = 0;
            for (int kb = 0; kb < nkb && !s_abort; ++kb) {
                kb_done = kb + 1;
                const int sb = kb & 1;
                if (!bar_wait(&b_empty[sb], (uint32_t)(((kb >> 1) & 1) ^ 1))) { s_abort = 1; break; }
                bar_expect(&b_full[sb], (uint32_t)L::B_SET);
                for (int t = 0; t < OZ_S; ++t)
                    tma2d(Bbuf + sb * L::B_SET + t * L::B_BYTES, &mapB, &b_full[sb], (kb0 + kb) * OZ_TK,
                          t * b_plane + b_row0 + n0);
                for (int s = 0; s < OZ_S; ++s, ++ia) {
                    const int sa = ia & 1;
                    if (!bar_wait(&a_empty[sa], (uint32_t)(((ia >> 1) & 1) ^ 1))) { s_abort = 1; break; }
                    bar_expect(&a_full[sa], (uint32_t)L::A_BYTES);
                    tma2d(Abuf + sa * L::A_BYTES, &mapA, &a_full[sa], (kb0 + kb) * OZ_TK, s * a_plane + a_row0 + m0);
                }
            }
            // every copy issued must land before the CTA can exit
            for (int kb = max(0, kb_done - 2); kb < kb_done; ++kb) bar_wait(&b_full[kb & 1], (uint32_t)((kb >> 1) & 1));
            for (int i = max(0, ia - 2); i < ia; ++i) bar_wait(&a_full[i & 1], (uint32_t)((i >> 1) & 1));
        }
    } else if (warp == 5) {
        if (lane == 0 && nkb > 0) {  // ---------------- MMA issuer
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                   ((uint32_t)(OZ_TM >> 4) << 24);
            int ia = 0, chunk = 0;
            for (int kb = 0; kb < nkb && !s_abort; ++kb) {
                const int sb = kb & 1;
                const bool first_of_chunk = (kb % OZ_CHUNK) == 0;
                if (first_of_chunk && chunk > 0) {
                    if (!bar_wait(c_free, (uint32_t)((chunk - 1) & 1))) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                if (!bar_wait(&b_full[sb], (uint32_t)((kb >> 1) & 1))) { s_abort = 1; break; }
                for (int s = 0; s < OZ_S; ++s, ++ia) {
                    const int sa = ia & 1;
                    if (!bar_wait(&a_full[sa], (uint32_t)((ia >> 1) & 1))) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = desc_sw128(su32(Abuf + sa * L::A_BYTES));
                    for (int t = 0; t + s < OZ_S; ++t) {
                        const uint64_t db = desc_sw128(su32(Bbuf + sb * L::B_SET + t * L::B_BYTES));
                        const uint32_t dt = tmem + (uint32_t)((s + t) * TN);
#pragma unroll
                        for (int k = 0; k < OZ_TK / 16; ++k) {
                            const uint64_t ko = (uint64_t)((k * 32) >> 4);
                            const uint32_t acc = (!first_of_chunk || s > 0 || k > 0) ? 1u : 0u;
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
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&b_empty[sb]))
                             : "memory");
                if ((kb % OZ_CHUNK) == OZ_CHUNK - 1 || kb == nkb - 1) {
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(c_full))
                                 : "memory");
                    ++chunk;
                }
            }
        }
    } else {  // ---------------- warps 0-3: drain TMEM into double-float
        float hi[TN], lo[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) hi[j] = lo[j] = 0.0f;
        bool ok = true;
        for (int ch = 0; ch < nchunks; ++ch) {
            ok = __all_sync(0xffffffffu, bar_wait(c_full, (uint32_t)(ch & 1)));
            if (!ok || s_abort) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int d = OZ_S - 1; d >= 0; --d) {
                const float w = __int_as_float((127 - 7 * (d + 2)) << 23);  // 2^{-7(d+2)}
#pragma unroll
                for (int c0 = 0; c0 < TN; c0 += 32) {
                    uint32_t v[32];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * TN + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float s, e;
                        two_sum(hi[c0 + j], __uint_as_float(v[j]) * w, s, e);
                        hi[c0 + j] = s;
                        lo[c0 + j] += e;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < TN; ++j) {  // renormalise (fast two-sum)
                float s = hi[j] + lo[j];
                lo[j] = lo[j] - (s - hi[j]);
                hi[j] = s;
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            bar_arrive(c_free);
        }
        if (!ok && lane == 0) atomicOr(status, ST_TIMEOUT);
        const int r = m0 + warp * 32 + lane;
        double* Pz = partial ? P + (size_t)blockIdx.z * (size_t)M * (size_t)N : nullptr;
        if (ok && !s_abort && r < M) {
            const int er = eA[r];
            // alpha = +-1 folds into the sign; beta in {0, 1} needs no multiply
            const bool unit_alpha = (alpha == 1.0 || alpha == -1.0);
            const unsigned long long sgn = (alpha < 0.0) ? (1ull << 63) : 0ull;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int c = n0 + j;
                if (c >= N) break;
                const int ec = eB[c];
                double v = 0.0;
                if (er != INT_MIN && ec != INT_MIN) {
                    double dh, dl;
                    if (unit_alpha && f32_to_f64_scaled(hi[j], er + ec, dh) && f32_to_f64_scaled(lo[j], er + ec, dl)) {
                        v = __longlong_as_double(__double_as_longlong(dh) ^ (long long)sgn) +
                            __longlong_as_double(__double_as_longlong(dl) ^ (long long)sgn);
                    } else {  // general alpha or extreme exponents
                        const double scale = ldexp(alpha, er + ec);
                        v = fma((double)hi[j], scale, (double)lo[j] * scale);
                    }
                }
                if (partial) {
                    Pz[r + (size_t)c * M] = v;
                } else {
                    double* cp = C + r + (int64_t)c * ldc;
                    *cp = (beta == 0.0) ? v : (beta == 1.0 ? *cp + v : fma(beta, *cp, v));
                }
            }
        }
    }
    if (s_abort && tid == 0) atomicOr(status, ST_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS) : "memory");
}

// C = sum_z P[z] (fixed order) + beta C
__global__ void k_oz_reduce(int M, int N, int S, const double* __restrict__ P, double beta, double* __restrict__ C,
                            int64_t ldc) {
    const int64_t total = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += P[(size_t)z * total + e];
        double* c = C + (e % M) + (e / M) * ldc;
        *c = (beta == 0.0) ? s : fma(beta, *c, s);
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

// short-K products with many output tiles (the rank-b updates) use 32-column
// tiles: 256 TMEM columns and ~97 KB of shared memory let two CTAs share an
// SM, so one's epilogue overlaps the other's MMAs
int oz_tn(int64_t M, int64_t N, int64_t K, int sms) {
    return (K <= 256 && cdiv(M, OZ_TM) * cdiv(N, 64) >= 4LL * sms) ? 32 : 64;
}

// split-K factor: slices of whole 128-deep chunks until the grid covers the
// SMs about twice; partials (FP64) need splits * M * N doubles
int oz_splits(int64_t M, int64_t N, int64_t K, int sms) {
    const int64_t tiles = cdiv(M, OZ_TM) * cdiv(N, oz_tn(M, N, K, sms));
    const int64_t chunks = cdiv(cdiv(K, OZ_TK), OZ_CHUNK);
    int64_t s = 1;
    if (tiles < 2LL * sms) s = cdiv(2LL * sms, tiles);
    if (s > chunks) s = chunks;
    if (s > 64) s = 64;
    if ((size_t)s * M * N > ((size_t)1 << 27)) s = 1;  // partials bounded at 1 GiB
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
                                                                                      status);
        k_oz_split<<<oz_grid(R * K), 256, 0, st>>>(X, ldx, (int)R, (int)K, true, e, Q, ldq);
    } else {
        k_oz_rowexp<<<(unsigned)cdiv(R, 32), 256, 0, st>>>(X, ldx, (int)R, (int)K, false, e, status);
        k_oz_split<<<dim3((unsigned)cdiv(R, 32), (unsigned)cdiv(K, 32)), 256, 0, st>>>(X, ldx, (int)R, (int)K, false,
                                                                                        e, Q, ldq);
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
    if (M < OZ_TM || N < OZ_TN || K < OZ_TK) return cudaErrorInvalidValue;  // one TMA box at least
    const int tn = oz_tn(M, N, K, sms);
    int splits = oz_splits(M, N, K, sms);
    if (sizeof(double) * (size_t)splits * M * N > p_bytes) splits = 1;
    CUtensorMap ma, mb;
    if (!oz_map(&ma, a.Q, (int64_t)OZ_S * a.plane, K, a.ldq, OZ_TM)) return cudaErrorInvalidValue;
    if (!oz_map(&mb, b.Q, (int64_t)OZ_S * b.plane, K, b.ldq, tn)) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             OzSmem<64>::TOTAL);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_oz_gemm<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     OzSmem<32>::TOTAL);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t nkb = cdiv(K, OZ_TK);
    const int kbs = (int)(cdiv(cdiv(nkb, OZ_CHUNK), splits) * OZ_CHUNK);  // whole chunks per split
    splits = (int)cdiv(nkb, kbs);
    dim3 grid((unsigned)cdiv(M, OZ_TM), (unsigned)cdiv(N, tn), (unsigned)splits);
    const int* eA = a.e + a_row0;
    const int* eB = b.e + b_row0;
    if (tn == 32)
        k_oz_gemm<32, 2><<<grid, OZ_THREADS, OzSmem<32>::TOTAL, st>>>(
            ma, mb, (int)M, (int)N, (int)K, eA, eB, alpha, beta, C, ldc, kbs, P, status, (int)a.plane, (int)a_row0,
            (int)b.plane, (int)b_row0);
    else
        k_oz_gemm<64, 1><<<grid, OZ_THREADS, OzSmem<64>::TOTAL, st>>>(
            ma, mb, (int)M, (int)N, (int)K, eA, eB, alpha, beta, C, ldc, kbs, P, status, (int)a.plane, (int)a_row0,
            (int)b.plane, (int)b_row0);
    trace_count(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    k_oz_reduce<<<oz_grid(M * N), 256, 0, st>>>((int)M, (int)N, splits, P, beta, C, ldc);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t oz_gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work, size_t work_bytes,
                    int sms, int* status, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (M < OZ_TM || N < OZ_TN || K < OZ_TK) return cudaErrorInvalidValue;  // one TMA box at least
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
