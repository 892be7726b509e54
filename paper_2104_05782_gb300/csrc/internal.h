// internal.h -- host-side launchers shared between the translation units of
// librandutv (C++ linkage, not exported).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>

namespace rutv {

// ---- FP64 DMMA products (gemm_f64.cu) --------------------------------------
// C = alpha op(A) op(B) + beta C (column-major).  partials (partial_elems
// doubles) enables the deterministic split-K for skinny products; may be null.
cudaError_t gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                     int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                     double* partials, size_t partial_elems, int sms, cudaStream_t st);
// Partial-buffer size (doubles) the split-K of an M x N x K product would use.
size_t gemm_f64_partial_elems(int64_t M, int64_t N, int64_t K, int sms);

// ---- Householder panel and compact WY factor (panel.cu) ---------------------
// Workspace (doubles) of panel_qr for a panel of width w on `grid` blocks.
size_t panel_qr_scratch_elems(int w, int grid);
// Number of blocks panel_qr launches for a panel of `len` rows.
int panel_qr_grid(int64_t len, int w, int sms);
// In-place Householder QR (dlarfg rule) of the len x w panel P (ld), tau[w].
// scratch: panel_qr_scratch_elems doubles; bar: one zeroed unsigned counter.
cudaError_t panel_qr(double* P, int64_t ld, int64_t len, int w, double* tau, double* scratch,
                     unsigned* bar, int* status, int sms, cudaStream_t st);
// W (len x w, ld len) := unit lower trapezoidal part of the QR storage P.
cudaError_t extract_w(const double* P, int64_t ld, int64_t len, int w, double* W, cudaStream_t st);
// Upper triangular Tf (w x w) of Q = I - W Tf W^T from Gram = W^T W and tau.
cudaError_t tfactor(const double* gram, const double* tau, int w, double* Tf, int* status,
                    cudaStream_t st);

// ---- b x b one-sided Jacobi SVD (svd.cu) ------------------------------------
size_t jacobi_scratch_elems(int w);
// SVD of the upper triangle of R (w x w, ldr): D (w), Us, Vs (w x w, ld w).
cudaError_t jacobi_svd(const double* R, int64_t ldr, int w, double* D, double* Us, double* Vs,
                       double* scratch, unsigned* bar, int* counters, int* status, int max_sweeps,
                       cudaStream_t st);

// ---- element-wise kernels (misc.cu) ---------------------------------------
cudaError_t gaussian_f64(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G, int64_t ldg,
                         cudaStream_t st);
cudaError_t set_identity(double* X, int64_t n, int64_t ld, cudaStream_t st);
cudaError_t copy_matrix(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                        cudaStream_t st);
// Block column T(k0:m, k0:k0+w) := [diag(D); 0].
cudaError_t set_diag_block(double* T, int64_t ldt, int64_t k0, int64_t m, int w, const double* D,
                           cudaStream_t st);
// *status |= ST_NONFINITE if any entry of the rows x cols matrix X is not finite.
cudaError_t check_finite(const double* X, int64_t ld, int64_t rows, int64_t cols, int* status,
                         cudaStream_t st);

}  // namespace rutv
