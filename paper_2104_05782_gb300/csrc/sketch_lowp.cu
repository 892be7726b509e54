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
                                float* __restrict__ X, DevGate gate) {
    if (gate_closed(gate)) return;
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
                                                float* __restrict__ Gp, DevGate gate) {
    if (gate_closed(gate)) return;
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

// G (b x b, upper triangle) = sum of the nparts partial Gram matrices, in a
// fixed order, spread over many blocks.
__global__ void k_gram_sum(const float* __restrict__ Gp, int nparts, int b, float* __restrict__ G, DevGate gate) {
    if (gate_closed(gate)) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e % b, j = e / b;
    float s = 0.0f;
    if (i <= j)
        for (int g = 0; g < nparts; ++g) s += Gp[(size_t)g * b * b + e];
    G[e] = s;
}

// Packed upper triangle: entry (p, c), p <= c, at c (c + 1) / 2 + p.
__device__ __forceinline__ int tri(int p, int c) { return c * (c + 1) / 2 + p; }
constexpr int CHOL_THREADS = 1024;

// One block: Cholesky G (+ shift) = R^T R of the upper triangle of G, with
// the triangle packed in shared memory (b (b + 1) / 2 floats; 132 KB at
// b = 256).  Right-looking: step j takes the pivot, then every warp updates
// whole columns c > j of the trailing triangle (lanes over its rows), reading
// row j unscaled and multiplying by 1 / pivot on the fly; row j itself is
// scaled during the next step, so each step needs two barriers.  A
// non-positive pivot (breakdown: numerically dependent columns) is replaced
// by the shift floor; the next pass repairs the basis.  R is written
// column-major b x b.
__global__ void __launch_bounds__(CHOL_THREADS) k_chol32(const float* __restrict__ G, int b, int L, int shift,
                                                         float* __restrict__ R, DevGate gate) {
    if (gate_closed(gate)) return;
    extern __shared__ float P[];
    __shared__ float s_tr, s_inv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = CHOL_THREADS / 32;
    for (int c = warp; c < b; c += NWARP)
        for (int p = lane; p <= c; p += 32) P[tri(p, c)] = G[p + (size_t)c * b];
    __syncthreads();
    if (tid == 0) {
        float tr = 0.0f;
        for (int i = 0; i < b; ++i) tr += P[tri(i, i)];
        s_tr = tr;
    }
    __syncthreads();
    const float u = 5.9604645e-8f;  // 2^-24
    const float sh = shift ? 11.0f * ((float)L * b + (float)b * (b + 1)) * u * s_tr : 0.0f;
    const float floor_ = fmaxf(sh, 1e-30f + u * s_tr);
    if (shift)
        for (int i = tid; i < b; i += CHOL_THREADS) P[tri(i, i)] += sh;
    __syncthreads();
    float inv_prev = 1.0f;
    for (int j = 0; j < b; ++j) {
        // row j - 1 scaled by its pivot's inverse (its last reader was step j - 1)
        if (j > 0)
            for (int c = j + tid; c < b; c += CHOL_THREADS) P[tri(j - 1, c)] *= inv_prev;
        if (tid == 0) {
            float d = P[tri(j, j)];
            if (!(d > 0.0f)) d = floor_;
            const float piv = sqrtf(d);
            P[tri(j, j)] = piv;
            s_inv = 1.0f / piv;
        }
        __syncthreads();
        const float inv = s_inv;
        for (int c = j + 1 + warp; c < b; c += NWARP) {
            const float rc = P[tri(j, c)] * inv;
            for (int p = j + 1 + lane; p <= c; p += 32) P[tri(p, c)] -= (P[tri(j, p)] * inv) * rc;
        }
        inv_prev = inv;
        __syncthreads();
    }
    // (row b - 1 holds only its pivot, so nothing is left to scale)
    for (int e = tid; e < b * b; e += CHOL_THREADS) {
        const int i = e % b, c = e / b;
        R[e] = (i <= c) ? P[tri(i, c)] : 0.0f;
    }
}

// X := X R^-1 (R upper b x b) for 32 rows per block: the rows' tile of X
// and the packed R sit in shared memory.  Columns go in blocks of 32: all
// threads first subtract the already solved blocks to the left
// (X_j -= X_{<j} R_{<j, j}, independent dot products), then one warp solves
// the 32 x 32 triangular block, a lane per row.  Optionally also writes the
// 16-bit K-major operand Xb[j*ldb + r].
constexpr int TRSM_ROWS = 32;
constexpr int TRSM_THREADS = 256;
constexpr int TRSM_LDX = TRSM_ROWS + 1;  // tile stride: lanes of a warp hit distinct banks
__global__ void __launch_bounds__(TRSM_THREADS) k_trsm32(float* __restrict__ X, int L, int b,
                                                         const float* __restrict__ R, uint16_t* __restrict__ Xb,
                                                         int64_t ldb, bool f16, DevGate gate) {
    if (gate_closed(gate)) return;
    extern __shared__ float tsm[];
    float* rs = tsm;                                // packed upper triangle of R
    float* xt = tsm + (size_t)b * (b + 1) / 2;      // TRSM_ROWS x b tile, column stride TRSM_LDX
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = blockIdx.x * TRSM_ROWS;
    const int nr = min(TRSM_ROWS, L - r0);
    for (int c = warp; c < b; c += TRSM_THREADS / 32)
        for (int p = lane; p <= c; p += 32) rs[tri(p, c)] = R[p + (size_t)c * b];
    for (int e = tid; e < TRSM_ROWS * b; e += TRSM_THREADS) {
        const int r = e % TRSM_ROWS, c = e / TRSM_ROWS;
        xt[r + TRSM_LDX * c] = (r < nr) ? X[(r0 + r) + (int64_t)c * L] : 0.0f;
    }
    __syncthreads();
    for (int jb = 0; jb < b; jb += 32) {
        const int wb = min(32, b - jb);
        if (jb > 0) {  // thread (r, q) updates columns jb + q + 8u of row r
            const int r = tid % TRSM_ROWS, q = tid / TRSM_ROWS;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int k = 0; k < jb; ++k) {
                const float xk = xt[r + TRSM_LDX * k];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = jb + q + 8 * u;
                    if (j < jb + wb) acc[u] = fmaf(xk, rs[tri(k, j)], acc[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jb + q + 8 * u;
                if (j < jb + wb) xt[r + TRSM_LDX * j] -= acc[u];
            }
        }
        __syncthreads();
        if (warp == 0) {
            for (int j = jb; j < jb + wb; ++j) {
                float s = xt[lane + TRSM_LDX * j];
                for (int k = jb; k < j; ++k) s = fmaf(-xt[lane + TRSM_LDX * k], rs[tri(k, j)], s);
                xt[lane + TRSM_LDX * j] = s / rs[tri(j, j)];
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < TRSM_ROWS * b; e += TRSM_THREADS) {
        const int r = e % TRSM_ROWS, c = e / TRSM_ROWS;
        if (r >= nr) continue;
        const float v = xt[r + TRSM_LDX * c];
        X[(r0 + r) + (int64_t)c * L] = v;
        if (Xb) Xb[(int64_t)c * ldb + r0 + r] = to16(v, f16);
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
    k_reduce_splits<<<grid_for(L * b), 256, 0, st>>>(P, stride, splits, (int)L, b, ldp, X, current_gate());
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
// the last pass also writes the 16-bit operand Xb (ld ldb).  b <= 256.
cudaError_t cholqr32(float* X, int64_t L, int b, int passes, uint16_t* Xb, int64_t ldb, bool f16, float* scratch,
                     int sms, cudaStream_t st) {
    if (L <= 0 || b <= 0) return cudaSuccess;
    if (b % 8 || b > 256) return cudaErrorInvalidValue;
    // partial Gram matrices over up to one block per SM, summed by many blocks
    int parts = (int)std::min<int64_t>(sms, cdiv(L, 128));
    parts = std::max(parts, 1);
    int chunk = (int)cdiv(L, parts);
    parts = (int)cdiv(L, chunk);
    float* Gp = scratch;
    float* G = scratch + (size_t)sms * b * b;
    float* R = G + (size_t)b * b;
    const size_t shm_tri = sizeof(float) * (size_t)b * (b + 1) / 2;
    const size_t shm_trsm = shm_tri + sizeof(float) * (size_t)TRSM_LDX * b;
    const size_t shm_gram = sizeof(float) * 32 * (size_t)b;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_gram32, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_chol32, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * 257 / 2 * 4);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_trsm32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (256 * 257 / 2 + TRSM_LDX * 256) * 4);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const DevGate gate = current_gate();
    for (int p = 0; p < passes; ++p) {
        {
            TraceScope ts("cholqr_gram", 2.0 * (double)L * b * b, 4.0 * (double)L * b, st);
            k_gram32<<<parts, 256, shm_gram, st>>>(X, (int)L, b, chunk, Gp, gate);
            k_gram_sum<<<(unsigned)cdiv((int64_t)b * b, 256), 256, 0, st>>>(Gp, parts, b, G, gate);
        }
        {
            TraceScope ts("cholqr_chol", (double)b * b * b / 3.0, 8.0 * (double)b * b, st);
            k_chol32<<<1, CHOL_THREADS, shm_tri, st>>>(G, b, (int)L, p == 0 ? 1 : 0, R, gate);
        }
        {
            TraceScope ts("cholqr_trsm", (double)L * b * b, 8.0 * (double)L * b, st);
            k_trsm32<<<(unsigned)cdiv(L, TRSM_ROWS), TRSM_THREADS, shm_trsm, st>>>(
                X, (int)L, b, R, p == passes - 1 ? Xb : nullptr, ldb, f16, gate);
        }
        trace_count(4);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace rutv
