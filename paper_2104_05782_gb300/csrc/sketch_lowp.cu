// sketch_lowp.cu -- element-wise and small dense kernels of the low-precision
// sketch (Sec. 3.2.1 with BF16 / scaled-FP16 operands):
//   - 16-bit shadows of T22 in the two K-major orientations the tcgen05
//     products need (S = T22 column-major for Y = T22^T X, St = T22 row-major
//     for Z = T22 Y), optionally scaled by a power of two (FP16 range);
//   - packing of FP64/FP32 column blocks (G, Y, Z) into 16-bit K-major
//     operands, reduction of split-K partials;
//   - FP32 re-orthonormalisation between products by shifted CholeskyQR
//     (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput.
//     2020): G = X^T X (+ s I on the first pass), G = R^T R, X := X R^-1,
//     three passes.  Re-orthonormalising keeps span(Y) in exact arithmetic,
//     so the sketch still spans (T22^T T22)^q T22^T G; it only keeps the
//     columns apart in low precision.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

__device__ __forceinline__ uint16_t to16(float v, bool f16) {
    if (f16) {
        __half h = __float2half_rn(v);
        return *reinterpret_cast<uint16_t*>(&h);
    }
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}

unsigned grid_for(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 8192)); }

// max |X| over a rows x cols FP64 matrix (non-negative doubles order like their
// bit patterns, so an integer atomicMax is exact and order independent).
__global__ void k_absmax(const double* __restrict__ X, int64_t ld, int64_t rows, int64_t cols,
                         unsigned long long* out) {
    int64_t total = rows * cols;
    double m = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        double v = fabs(X[i + j * ld]);
        m = v > m ? v : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        double t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// FP16 scale 2^e with 2^e * max|T22| in [2^13, 2^14): keeps every product of the
// scaled shadow (|.| <= 2^14) and an orthonormal column (|.| <= 1) inside FP16
// range.  BF16 uses scale 1.
__device__ __forceinline__ float shadow_scale(const unsigned long long* amax, bool f16) {
    if (!f16 || amax == nullptr) return 1.0f;
    double m = __longlong_as_double((long long)*amax);
    if (!(m > 0.0) || !isfinite(m)) return 1.0f;
    int e;
    frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
    return ldexpf(1.0f, 14 - e);
}

// S(i, k) = s T22(k, i) -> S[i*lds + k]   (rows = m', cols = n' of T22)
// St(k', i') = s T22(k', i')  -> St[k'*ldst + i']
__global__ void k_shadow(const double* __restrict__ T22, int64_t ldt, int rows, int cols, uint16_t* __restrict__ S,
                         int64_t lds, uint16_t* __restrict__ St, int64_t ldst, bool f16,
                         const unsigned long long* amax) {
    __shared__ float tile[32][33];
    const float s = shadow_scale(amax, f16);
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        int r = r0 + tx, c = c0 + j;
        float v = 0.0f;
        if (r < rows && c < cols) v = (float)(T22[r + (int64_t)c * ldt] * (double)s);
        tile[j][tx] = v;  // tile[col][row]
        if (r < rows && c < cols) S[(int64_t)c * lds + r] = to16(v, f16);
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        int r = r0 + j, c = c0 + tx;
        if (r < rows && c < cols) St[(int64_t)r * ldst + c] = to16(tile[tx][j], f16);
    }
}

// 16-bit K-major operand: Xb[j*ldb + k] = X(k, j) for k < L, j < b (FP64 or FP32 source).
template <typename T>
__global__ void k_pack16(const T* __restrict__ X, int64_t ldx, int L, int b, uint16_t* __restrict__ Xb, int64_t ldb,
                         bool f16) {
    int64_t total = (int64_t)L * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = e % L, j = e / L;
        Xb[j * ldb + k] = to16((float)X[k + j * ldx], f16);
    }
}

// X(r, c) = sum_z P[z](r, c) for r < L, c < b (fixed order), column-major ld L.
__global__ void k_reduce_splits(const float* __restrict__ P, int64_t stride, int splits, int L, int b, int64_t ldp,
                                float* __restrict__ X) {
    int64_t total = (int64_t)L * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % L, c = e / L;
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += P[z * stride + r + c * ldp];
        X[r + c * L] = s;
    }
}

__global__ void k_f32_to_f64(const float* __restrict__ X, int64_t total, double* __restrict__ Y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = (double)X[e];
}

// Partial Gram matrices: block g sums rows [g*chunk, (g+1)*chunk) of X^T X.
// 8 x 8 register micro-tiles over (p, q), rows staged through shared memory.
__global__ void __launch_bounds__(256) k_gram32(const float* __restrict__ X, int L, int b, int chunk,
                                                float* __restrict__ Gp) {
    extern __shared__ float xs[];  // 32 rows x b
    const int r0 = blockIdx.x * chunk, r1 = min(L, r0 + chunk);
    const int nt = (b / 8) * (b / 8);
    float* out = Gp + (size_t)blockIdx.x * b * b;
    for (int t0 = 0; t0 < nt; t0 += 256) {
        const int t = t0 + threadIdx.x;
        const int p0 = (t / (b / 8)) * 8, q0 = (t % (b / 8)) * 8;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
        for (int rb = r0; rb < r1; rb += 32) {
            const int nr = min(32, r1 - rb);
            __syncthreads();
            for (int e = threadIdx.x; e < 32 * b; e += 256) {
                int rr = e % 32, c = e / 32;
                xs[rr * b + c] = (rr < nr) ? X[(rb + rr) + (int64_t)c * L] : 0.0f;
            }
            __syncthreads();
            if (t < nt) {
                for (int rr = 0; rr < nr; ++rr) {
                    float a[8], bb[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) a[i] = xs[rr * b + p0 + i];
#pragma unroll
                    for (int j = 0; j < 8; ++j) bb[j] = xs[rr * b + q0 + j];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
                }
            }
        }
        if (t < nt)
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) out[(p0 + i) + (size_t)(q0 + j) * b] = acc[i][j];
    }
}

// One block: G = sum of partials (+ shift) and its Cholesky factor G = R^T R
// (upper R), written column-major b x b to R.  A non-positive pivot
// (breakdown: the columns were numerically dependent) is replaced by the
// shift floor; the next pass repairs the basis.  G lives in shared memory
// when it fits (b <= 128), else in the global scratch Gg.
__global__ void __launch_bounds__(256) k_chol32(const float* __restrict__ Gp, int nparts, int b, int L, int shift,
                                                float* __restrict__ Gg, float* __restrict__ R, int use_smem) {
    extern __shared__ float csm[];
    __shared__ float s_tr, s_piv;
    float* G = use_smem ? csm : Gg;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < b * b; e += nt) {
        const int i = e % b, j = e / b;
        float s = 0.0f;
        if (i <= j)
            for (int g = 0; g < nparts; ++g) s += Gp[(size_t)g * b * b + e];
        G[e] = s;
    }
    __syncthreads();
    if (tid == 0) {
        float tr = 0.0f;
        for (int i = 0; i < b; ++i) tr += G[i + (size_t)i * b];
        s_tr = tr;
    }
    __syncthreads();
    const float u = 5.9604645e-8f;  // 2^-24
    const float sh = shift ? 11.0f * ((float)L * b + (float)b * (b + 1)) * u * s_tr : 0.0f;
    const float floor_ = fmaxf(sh, 1e-30f + u * s_tr);
    if (shift)
        for (int i = tid; i < b; i += nt) G[i + (size_t)i * b] += sh;
    __syncthreads();
    // right-looking Cholesky on the upper triangle: row j of R overwrites row j of G
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            float d = G[j + (size_t)j * b];
            if (!(d > 0.0f)) d = floor_;
            s_piv = sqrtf(d);
        }
        __syncthreads();
        const float piv = s_piv, inv = 1.0f / piv;
        // trailing update, one column per thread (row j scaled on the fly)
        for (int c = j + 1 + tid; c < b; c += nt) {
            float* gc = G + (size_t)c * b;
            const float rc = gc[j] * inv;
            for (int p = j + 1; p <= c; ++p) gc[p] -= (G[j + (size_t)p * b] * inv) * rc;
        }
        __syncthreads();
        for (int c = j + 1 + tid; c < b; c += nt) G[j + (size_t)c * b] *= inv;
        if (tid == 0) G[j + (size_t)j * b] = piv;
        __syncthreads();
    }
    for (int e = tid; e < b * b; e += nt) {
        const int i = e % b, j = e / b;
        R[e] = (i <= j) ? G[e] : 0.0f;
    }
}

// X := X R^-1 (R upper b x b) by forward substitution, one row per thread;
// optionally also writes the 16-bit K-major operand Xb[j*ldb + r].
__global__ void __launch_bounds__(128) k_trsm32(float* __restrict__ X, int L, int b, const float* __restrict__ R,
                                                uint16_t* __restrict__ Xb, int64_t ldb, bool f16, int use_smem) {
    extern __shared__ float rs[];
    const float* Rr = R;
    if (use_smem) {
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) rs[e] = R[e];
        __syncthreads();
        Rr = rs;
    }
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= L) return;
    for (int j = 0; j < b; ++j) {
        float s = X[r + (int64_t)j * L];
        const float* rc = Rr + (size_t)j * b;
        for (int k = 0; k < j; ++k) s = fmaf(-X[r + (int64_t)k * L], rc[k], s);
        s /= rc[j];
        X[r + (int64_t)j * L] = s;
        if (Xb) Xb[(int64_t)j * ldb + r] = to16(s, f16);
    }
}

}  // namespace

cudaError_t absmax_f64(const double* X, int64_t ld, int64_t rows, int64_t cols, unsigned long long* out,
                       cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || rows <= 0 || cols <= 0) return e;
    k_absmax<<<std::min<unsigned>(grid_for(rows * cols), 1024), 256, 0, st>>>(X, ld, rows, cols, out);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t shadow16(const double* T22, int64_t ldt, int64_t rows, int64_t cols, uint16_t* S, int64_t lds,
                     uint16_t* St, int64_t ldst, bool f16, const unsigned long long* amax, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((unsigned)cdiv(rows, 32), (unsigned)cdiv(cols, 32));
    k_shadow<<<grid, dim3(32, 8), 0, st>>>(T22, ldt, (int)rows, (int)cols, S, lds, St, ldst, f16, f16 ? amax : nullptr);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t pack16_f64(const double* X, int64_t ldx, int64_t L, int b, uint16_t* Xb, int64_t ldb, bool f16,
                       cudaStream_t st) {
    if (L <= 0 || b <= 0) return cudaSuccess;
    k_pack16<double><<<grid_for(L * b), 256, 0, st>>>(X, ldx, (int)L, b, Xb, ldb, f16);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t reduce_splits(const float* P, int64_t stride, int splits, int64_t L, int b, int64_t ldp, float* X,
                          cudaStream_t st) {
    if (L <= 0 || b <= 0) return cudaSuccess;
    k_reduce_splits<<<grid_for(L * b), 256, 0, st>>>(P, stride, splits, (int)L, b, ldp, X);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t f32_to_f64(const float* X, int64_t total, double* Y, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_f32_to_f64<<<grid_for(total), 256, 0, st>>>(X, total, Y);
    trace_count(1);
    return cudaGetLastError();
}

size_t cholqr_scratch_floats(int b, int sms) { return (size_t)(sms + 1) * b * b + 2 * (size_t)b * b; }

// Shifted CholeskyQR, `passes` passes, on X (L x b FP32, column-major ld L);
// the last pass also writes the 16-bit operand Xb (ld ldb).
cudaError_t cholqr32(float* X, int64_t L, int b, int passes, uint16_t* Xb, int64_t ldb, bool f16, float* scratch,
                     int sms, cudaStream_t st) {
    if (L <= 0 || b <= 0) return cudaSuccess;
    if (b % 8) return cudaErrorInvalidValue;
    // few partial Gram matrices keep the single-block reduction short
    int parts = (int)std::min<int64_t>(std::min(sms, 48), cdiv(L, 256));
    parts = std::max(parts, 1);
    int chunk = (int)cdiv(L, parts);
    parts = (int)cdiv(L, chunk);
    float* Gp = scratch;
    float* G = scratch + (size_t)sms * b * b;
    float* R = G + (size_t)b * b;
    const int small = (b <= 128) ? 1 : 0;
    const size_t shm_chol = small ? sizeof(float) * (size_t)b * b : 0;
    const size_t shm_trsm = small ? sizeof(float) * (size_t)b * b : 0;
    const size_t shm_gram = sizeof(float) * 32 * (size_t)b;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_gram32, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        cudaFuncSetAttribute(k_chol32, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4);
        cudaFuncSetAttribute(k_trsm32, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4);
        configured = true;
    }
    for (int p = 0; p < passes; ++p) {
        {
            TraceScope ts("cholqr_gram", 2.0 * (double)L * b * b, 4.0 * (double)L * b, st);
            k_gram32<<<parts, 256, shm_gram, st>>>(X, (int)L, b, chunk, Gp);
        }
        {
            TraceScope ts("cholqr_chol", (double)b * b * b / 3.0, 4.0 * (double)parts * b * b, st);
            k_chol32<<<1, 256, shm_chol, st>>>(Gp, parts, b, (int)L, p == 0 ? 1 : 0, G, R, small);
        }
        {
            TraceScope ts("cholqr_trsm", (double)L * b * b, 8.0 * (double)L * b, st);
            k_trsm32<<<(unsigned)cdiv(L, 128), 128, shm_trsm, st>>>(X, (int)L, b, R, p == passes - 1 ? Xb : nullptr,
                                                                      ldb, f16, small);
        }
        trace_count(3);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rutv
