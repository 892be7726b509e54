// gemm_f64.cu -- FP64 matrix products on the DMMA tensor path (mma.sync f64).
//
// Every FP64 product of the randUTV step runs here: the sketch and power
// iteration Y = T22^T G, Z = T22 Y (Sec. 3.2.1), the three products of each
// compact-WY application C - (C W) T W^T and C - W T^T (W^T C) (Sec. 2.3,
// Sec. 5.4 "applying V_alpha / U_alpha"), the Gram matrix W^T W of the
// triangular factor, and the b x b products of the small SVD (Sec. 3.2.3).
//
// GB300 has no tcgen05 kind for f64, and its FP64 rate is ~1.05 TFLOP/s
// whether issued as DFMA or as mma.sync.m8n8k4.f64 (both measured).  At that
// rate every product here is compute bound by two orders of magnitude (a
// 64x64x16 tile does 131k flop per 16 KB staged), so the kernel is built for
// issue efficiency and load balance rather than for data movement: 64x64 CTA
// tiles, four warps of 32x32 (16 independent m8n8k4 MMAs per k-step), a
// register-prefetched shared-memory stage, and a deterministic split-K
// (partials summed in a fixed order) for the skinny products whose tile count
// would otherwise leave SMs idle in the last wave.
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NTHREADS = 128;
constexpr int APAD = 2, BPAD = 2;

__device__ __forceinline__ void dmma884(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// C(M x N) = alpha * op(A) op(B) + beta * C, column-major.
// op(A)(i,k) = TA ? A[k + i*lda] : A[i + k*lda];  op(B)(k,j) = TB ? B[j + k*ldb] : B[k + j*ldb].
// gridDim.z > 1: slice z covers k in [z*kchunk, (z+1)*kchunk) and writes
// alpha * partial into P + z*M*N (ld M) instead of C.
template <bool TA, bool TB>
__global__ void __launch_bounds__(NTHREADS) k_gemm_f64(int M, int N, int K, double alpha,
                                                       const double* __restrict__ A, int64_t lda,
                                                       const double* __restrict__ B, int64_t ldb,
                                                       double beta, double* __restrict__ C, int64_t ldc,
                                                       double* __restrict__ P, int kchunk, DevGate gate) {
    if (gate_closed(gate)) return;
    __shared__ double As[BK][BM + APAD];
    __shared__ double Bs[BK][BN + BPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;

    double acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    double ra[8], rb[8];
    auto load_tile = [&](int k0) {
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            int idx = tid + it * NTHREADS;
            int m, k;
            if (!TA) { m = idx % BM; k = idx / BM; } else { k = idx % BK; m = idx / BK; }
            int gi = row0 + m, gk = k0 + k;
            double v = 0.0;
            if (gi < M && gk < kend) v = TA ? A[gk + (int64_t)gi * lda] : A[gi + (int64_t)gk * lda];
            ra[it] = v;
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            int idx = tid + it * NTHREADS;
            int n, k;
            if (TB) { n = idx % BN; k = idx / BN; } else { k = idx % BK; n = idx / BK; }
            int gj = col0 + n, gk = k0 + k;
            double v = 0.0;
            if (gj < N && gk < kend) v = TB ? B[gj + (int64_t)gk * ldb] : B[gk + (int64_t)gj * ldb];
            rb[it] = v;
        }
    };
    auto store_tile = [&]() {
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            int idx = tid + it * NTHREADS;
            int m, k;
            if (!TA) { m = idx % BM; k = idx / BM; } else { k = idx % BK; m = idx / BK; }
            As[k][m] = ra[it];
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            int idx = tid + it * NTHREADS;
            int n, k;
            if (TB) { n = idx % BN; k = idx / BN; } else { k = idx % BK; n = idx / BK; }
            Bs[k][n] = rb[it];
        }
    };

    if (kbeg < kend) {
        load_tile(kbeg);
        for (int k0 = kbeg; k0 < kend; k0 += BK) {
            __syncthreads();
            store_tile();
            __syncthreads();
            if (k0 + BK < kend) load_tile(k0 + BK);
#pragma unroll
            for (int kk = 0; kk < BK; kk += 4) {
                double af[4], bf[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) af[i] = As[kk + (lane & 3)][wm + i * 8 + (lane >> 2)];
#pragma unroll
                for (int j = 0; j < 4; ++j) bf[j] = Bs[kk + (lane & 3)][wn + j * 8 + (lane >> 2)];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) dmma884(acc[i][j], af[i], bf[j]);
            }
        }
    }

    // epilogue: fragment (i,j) holds rows wm+8i+(lane>>2), cols wn+8j+2(lane&3)+{0,1}
    const bool partial = (gridDim.z > 1);
    double* Pz = partial ? P + (size_t)blockIdx.z * (size_t)M * (size_t)N : nullptr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gi = row0 + wm + i * 8 + (lane >> 2);
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int gj = col0 + wn + j * 8 + 2 * (lane & 3) + h;
                if (gj >= N) continue;
                double v = alpha * acc[i][j][h];
                if (partial) {
                    Pz[gi + (size_t)gj * M] = v;
                } else {
                    double* c = C + gi + (int64_t)gj * ldc;
                    *c = (beta == 0.0) ? v : v + beta * (*c);
                }
            }
        }
    }
}

// C = sum_z P[z] (fixed order z = 0..S-1) + beta * C.
__global__ void k_splitk_reduce(int M, int N, int S, const double* __restrict__ P, double beta,
                                double* __restrict__ C, int64_t ldc, DevGate gate) {
    if (gate_closed(gate)) return;
    int64_t total = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(e % M);
        int64_t j = e / M;
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += P[(size_t)z * total + e];
        double* c = C + i + j * ldc;
        *c = (beta == 0.0) ? s : s + beta * (*c);
    }
}

}  // namespace

size_t gemm_f64_partial_elems(int64_t M, int64_t N, int64_t K, int sms) {
    int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
    if (tiles <= 0 || K <= 0) return 0;
    int64_t target = 8LL * sms;
    if (tiles >= target) return 0;
    int64_t S = cdiv(target, tiles);
    int64_t smax = K / 256;
    if (S > smax) S = smax;
    if (S <= 1) return 0;
    return (size_t)(S * M * N);
}

cudaError_t gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                     int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                     double* partials, size_t partial_elems, int sms, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0) {  // C = beta * C
        if (beta == 1.0) return cudaSuccess;
        k_splitk_reduce<<<(unsigned)std::min<int64_t>(cdiv(M * N, 256), 4096), 256, 0, st>>>(
            (int)M, (int)N, 0, partials, beta, C, ldc, current_gate());
        trace_count(1);
        return cudaGetLastError();
    }
    int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
    int64_t target = 8LL * sms;
    int S = 1;
    if (tiles < target && partials != nullptr) {
        int64_t s = cdiv(target, tiles);
        int64_t smax = K / 256;
        if (s > smax) s = smax;
        while (s > 1 && (size_t)(s * M * N) > partial_elems) --s;
        if (s > 1) S = (int)s;
    }
    int kchunk = (int)(cdiv(cdiv(K, S), BK) * BK);
    S = (int)cdiv(K, kchunk);
    dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)S);
    dim3 block(NTHREADS);
#define LAUNCH(TA_, TB_)                                                                             \
    k_gemm_f64<TA_, TB_><<<grid, block, 0, st>>>((int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, \
                                                 C, ldc, partials, kchunk, current_gate())
    if (!ta && !tb) LAUNCH(false, false);
    else if (ta && !tb) LAUNCH(true, false);
    else if (!ta && tb) LAUNCH(false, true);
    else LAUNCH(true, true);
#undef LAUNCH
    trace_count(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S == 1) return e;
    int64_t total = M * N;
    unsigned blocks = (unsigned)std::min<int64_t>(cdiv(total, 256), 8LL * sms);
    k_splitk_reduce<<<blocks, 256, 0, st>>>((int)M, (int)N, S, partials, beta, C, ldc, current_gate());
    trace_count(1);
    return cudaGetLastError();
}

}  // namespace rutv
