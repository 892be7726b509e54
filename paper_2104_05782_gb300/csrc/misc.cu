// misc.cu -- element-wise kernels of the randUTV step: the Gaussian draw of the
// sketch, identity initialisation, strided copies, the diagonal block write and
// the finiteness check.
#include "common.cuh"
#include "internal.h"
#include "trace.h"
#include "philox.cuh"

namespace rutv {

namespace {

// G^(step)(r, c) of Sec. 3.2.1 (see gaussian4).
__global__ void k_gaussian(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* __restrict__ G,
                           int64_t ldg) {
    const int64_t groups = (rows + 3) / 4;
    const int64_t total = groups * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = e % groups, c = e / groups;
        double z[4];
        gaussian4(seed, step, k, c, z);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int64_t r = 4 * k + t;
            if (r < rows) G[r + c * ldg] = z[t];
        }
    }
}

__global__ void k_set_identity(double* __restrict__ X, int64_t n, int64_t ld) {
    int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % n, j = e / n;
        X[i + j * ld] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void k_set_eye_rect(double* __restrict__ X, int64_t rows, int64_t cols, int64_t ld) {
    int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        X[i + j * ld] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void k_copy(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
                       int64_t rows, int64_t cols) {
    int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        dst[i + j * ldd] = src[i + j * lds];
    }
}

__global__ void k_set_diag_block(double* __restrict__ T, int64_t ldt, int64_t k0, int64_t m, int w,
                                 const double* __restrict__ D) {
    int64_t rows = m - k0;
    int64_t total = rows * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        T[(k0 + i) + (k0 + j) * ldt] = (i == j) ? D[j] : 0.0;
    }
}

__global__ void k_check_finite(const double* __restrict__ X, int64_t ld, int64_t rows, int64_t cols, int* status) {
    int64_t total = rows * cols;
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        bad |= !isfinite(X[i + j * ld]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
}

// X(i, j) := 0 below the diagonal (i > j) of a rows x cols matrix.
__global__ void k_zero_below(double* __restrict__ X, int64_t ld, int64_t rows, int64_t cols) {
    int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % rows, j = e / rows;
        if (i > j) X[i + j * ld] = 0.0;
    }
}

// X (m x m) := diag(X(0:n, 0:n), I_{m-n}): every entry outside the leading
// n x n block is set to the identity's.
__global__ void k_embed_identity(double* __restrict__ X, int64_t ld, int64_t m, int64_t n) {
    int64_t total = m * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e % m, j = e / m;
        if (i >= n || j >= n) X[i + j * ld] = (i == j) ? 1.0 : 0.0;
    }
}

// Flat copies by the SMs (dst, src 16- or 8-byte aligned): used between
// pinned host memory and the device, where they keep the link's full rate
// even after it has been idle (DMA copies were measured an order of
// magnitude slower then).
__global__ void k_copy16(const double2* __restrict__ src, double2* __restrict__ dst, int64_t n2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
__global__ void k_copy8(const double* __restrict__ src, double* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

unsigned grid_for(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 8192)); }

}  // namespace

cudaError_t gaussian_f64(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G, int64_t ldg,
                         cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    k_gaussian<<<grid_for(cdiv(rows, 4) * cols), 256, 0, st>>>(seed, step, rows, cols, G, ldg);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t set_identity(double* X, int64_t n, int64_t ld, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_set_identity<<<grid_for(n * n), 256, 0, st>>>(X, n, ld);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t set_eye_rect(double* X, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    k_set_eye_rect<<<grid_for(rows * cols), 256, 0, st>>>(X, rows, cols, ld);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t copy_matrix(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                        cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    k_copy<<<grid_for(rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t set_diag_block(double* T, int64_t ldt, int64_t k0, int64_t m, int w, const double* D,
                           cudaStream_t st) {
    if (w <= 0 || m - k0 <= 0) return cudaSuccess;
    k_set_diag_block<<<grid_for((m - k0) * w), 256, 0, st>>>(T, ldt, k0, m, w, D);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t copy_flat(const double* src, double* dst, int64_t count, int sms, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::max(1, 4 * sms);
    if (((uintptr_t)src | (uintptr_t)dst) % 16 == 0) {
        const int64_t n2 = count / 2;
        if (n2 > 0) k_copy16<<<blocks, 512, 0, st>>>((const double2*)src, (double2*)dst, n2);
        if (count % 2) k_copy8<<<1, 32, 0, st>>>(src + 2 * n2, dst + 2 * n2, 1);
    } else {
        k_copy8<<<blocks, 512, 0, st>>>(src, dst, count);
    }
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t zero_below_diag(double* X, int64_t ld, int64_t rows, int64_t cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    k_zero_below<<<grid_for(rows * cols), 256, 0, st>>>(X, ld, rows, cols);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t embed_identity(double* X, int64_t ld, int64_t m, int64_t n, cudaStream_t st) {
    if (m <= 0 || m == n) return cudaSuccess;
    k_embed_identity<<<grid_for(m * m), 256, 0, st>>>(X, ld, m, n);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t check_finite(const double* X, int64_t ld, int64_t rows, int64_t cols, int* status, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    k_check_finite<<<grid_for(rows * cols), 256, 0, st>>>(X, ld, rows, cols, status);
    trace_count(1);
    return cudaGetLastError();
}

}  // namespace rutv
