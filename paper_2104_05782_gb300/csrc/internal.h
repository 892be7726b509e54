// internal.h -- host-side launchers shared between the translation units of
// librandutv (C++ linkage, not exported).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>

namespace rutv {

// ---- launch gate of the product kernels (randutv.cu) -------------------------
// The product, split and reduction launchers below pass the calling thread's
// current gate (DevGate of common.cuh) to their kernels; a GateScope sets it
// for the launches made during its lifetime.
struct DevGate;
const DevGate& current_gate();
class GateScope {
  public:
    GateScope(const int* flag, int need);
    ~GateScope();
    GateScope(const GateScope&) = delete;
    GateScope& operator=(const GateScope&) = delete;

  private:
    const int* saved_flag_;
    int saved_need_;
};

// ---- process-wide limits of the device-side failure detection (randutv.cu) --
// Polls after which a grid barrier gives up (ST_TIMEOUT), and the sweep cap
// of the b x b Jacobi SVD (ST_NOCONV).  Defaults: kSpinLimit and 30.
long long wait_limit();
int sweep_cap();

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
// Same factorization for w <= 32, which also writes the compact WY form of
// the panel: W (len x w, ld len, as extract_w) and Tf (w x w, ld w, as tfactor
// of W^T W), the Gram matrix formed inside the kernel.
cudaError_t panel_qr_wy(double* P, int64_t ld, int64_t len, int w, double* tau, double* W, double* Tf,
                        double* scratch, unsigned* bar, int* status, int sms, cudaStream_t st);
// W (len x w, ld len) := unit lower trapezoidal part of the QR storage P.
cudaError_t extract_w(const double* P, int64_t ld, int64_t len, int w, double* W, cudaStream_t st);
// Upper triangular Tf (w x w, ld w) of Q = I - W Tf W^T from Gram = W^T W and tau.
cudaError_t tfactor(const double* gram, const double* tau, int w, double* Tf, int* status,
                    cudaStream_t st);

// ---- b x b one-sided Jacobi SVD (svd.cu) ------------------------------------
size_t jacobi_scratch_elems(int w);
// SVD of the upper triangle of R (w x w, ldr): D (w), Us, Vs (w x w, ld w).
// allow_cluster = false forces the grid variant that works in `scratch`.
// dense: use all of R (not only its upper triangle); V0 (w x w, ld w, or
// null for I): starting V, so that Vs = V0 W for the rotations W applied.
cudaError_t jacobi_svd(const double* R, int64_t ldr, int w, double* D, double* Us, double* Vs,
                       double* scratch, unsigned* bar, int* counters, int* status, int max_sweeps,
                       cudaStream_t st, bool allow_cluster = true, bool dense = false,
                       const double* V0 = nullptr);
// FP32 Jacobi on the upper triangle of R (w <= 128): its accumulated right
// rotations, orthogonal to FP32 accuracy, as FP64 Q0 (w x w, ld w).
cudaError_t jacobi32_precondition(const double* R, int64_t ldr, int w, double* Q0, int max_sweeps, cudaStream_t st);
// U (w x w, ld w) := upper triangle of R.
cudaError_t triu_copy(const double* R, int64_t ldr, int w, double* U, cudaStream_t st);

// ---- element-wise kernels (misc.cu) ---------------------------------------
cudaError_t gaussian_f64(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G, int64_t ldg,
                         cudaStream_t st);
cudaError_t set_identity(double* X, int64_t n, int64_t ld, cudaStream_t st);
cudaError_t copy_matrix(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                        cudaStream_t st);
// Block column T(k0:m, k0:k0+w) := [diag(D); 0].
cudaError_t set_diag_block(double* T, int64_t ldt, int64_t k0, int64_t m, int w, const double* D,
                           cudaStream_t st);
// dst[0:count) := src[0:count) by the SMs (either may be pinned host memory
// given by its device address).
cudaError_t copy_flat(const double* src, double* dst, int64_t count, int sms, cudaStream_t st);
// X(i, j) := 0 for i > j (rows x cols).
cudaError_t zero_below_diag(double* X, int64_t ld, int64_t rows, int64_t cols, cudaStream_t st);
// X (m x m) := diag(X(0:n, 0:n), I_{m-n}).
cudaError_t embed_identity(double* X, int64_t ld, int64_t m, int64_t n, cudaStream_t st);
// *status |= ST_NONFINITE if any entry of the rows x cols matrix X is not finite.
cudaError_t check_finite(const double* X, int64_t ld, int64_t rows, int64_t cols, int* status,
                         cudaStream_t st);

// ---- low-precision sketch (tc_gemm.cu, sketch_lowp.cu) ------------------------
int tc_gemm_npad(int Nb);
int tc_gemm_splits(int64_t M, int64_t K, int sms);
cudaError_t tc_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int Nb, int64_t K, bool f16,
                    float* C, int64_t ldc, int64_t split_stride, int splits, int* status, cudaStream_t st);
cudaError_t absmax_f64(const double* X, int64_t ld, int64_t rows, int64_t cols, unsigned long long* out,
                       cudaStream_t st);
cudaError_t shadow16(const double* T22, int64_t ldt, int64_t rows, int64_t cols, uint16_t* S, int64_t lds,
                     uint16_t* St, int64_t ldst, bool f16, const unsigned long long* amax, cudaStream_t st);
cudaError_t pack16_f64(const double* X, int64_t ldx, int64_t L, int b, uint16_t* Xb, int64_t ldb, bool f16,
                       cudaStream_t st);
cudaError_t reduce_splits(const float* P, int64_t stride, int splits, int64_t L, int b, int64_t ldp, float* X,
                          cudaStream_t st);
cudaError_t f32_to_f64(const float* X, int64_t total, double* Y, cudaStream_t st);
size_t cholqr_scratch_floats(int b, int sms);
cudaError_t cholqr32(float* X, int64_t L, int b, int passes, uint16_t* Xb, int64_t ldb, bool f16, float* scratch,
                     int sms, cudaStream_t st);

// ---- learned q (learnq.cu) --------------------------------------------------
int learnq_nparam();
// Features of a block step from the previous block's diagonal (dprev[j * dstride],
// j < wprev; wprev = 0 for the first block of the call) and the QR storage R of
// the compressed q = 0 sketch.  lvl[0]: the sketch's Frobenius norm when
// have_level (else formed from R), lvl[1]: the first block's, kept here.
cudaError_t learnq_features(const double* dprev, int64_t dstride, int wprev, const double* R, int64_t ldr, int w,
                            float* f, double* lvl, bool have_level, cudaStream_t st);
// E (e x w, ld e) := S Y with S the CountSketch r -> r mod e, sign from a
// hash of key + r (Y: L x w, ld ldy).
cudaError_t countsketch(const double* Y, int64_t ldy, int64_t L, int w, int e, uint64_t key, double* E,
                        cudaStream_t st);
// rdiag (w doubles) := |R_jj| of the Householder QR of E (e x w, ld lde) in
// FP32 in one block; *level := ||E||_F (FP64); e <= 256, w <= 128.
cudaError_t feature_rdiag(const double* E, int64_t lde, int e, int w, double* rdiag, double* level,
                          cudaStream_t st);
// q (device) := the network's choice; also written to *qlog when qlog != null.
cudaError_t learnq_infer(const float* P, const float* f, int fallback, int* q, int* qlog, cudaStream_t st);
size_t learnq_train_scratch_floats(int N);
cudaError_t learnq_train_step(float* P, const float* X, const int* y, int N, float* scratch, float* grads_out,
                              float* loss_out, int t, float lr, float wd, cudaStream_t st);
cudaError_t learnq_predict(const float* P, const float* X, int N, float* probs, cudaStream_t st);
// ---- FP64 products emulated on BF16 tensor cores (oz_gemm.cu) ---------------
int64_t oz_ldq(int64_t K);
size_t oz_work_bytes(int64_t M, int64_t N, int64_t K);
// One operand split into OZ_S = 8 BF16 digit planes with a power-of-two
// scale per row: L(r, k) = trans ? X(k, r) : X(r, k), r < R, k < K.  Plane s
// holds rows [s * plane, s * plane + R) of a row-major array with ldq BF16
// per row; e[r] is the row's scale exponent.
struct OzOperand {
    const uint16_t* Q;
    const int* e;
    int64_t R, K, plane, ldq;
};
size_t oz_operand_bytes(int64_t R, int64_t K);
// Splits X into `buf` (oz_operand_bytes(R, K) bytes, 256-byte aligned).
cudaError_t oz_split(bool trans, const double* X, int64_t ldx, int64_t R, int64_t K, void* buf, OzOperand* out,
                     int* status, cudaStream_t st);
// C (M x N) = alpha La(a_row0 : a_row0 + M, :) Lb(b_row0 : b_row0 + N, :)^T + beta C
// from split operands; needs operands of at least 16 (La) and 4 (Lb) rows,
// and, when K < 64, both split with the same ldq; P holds the FP64 split-K
// partials (p_bytes bytes; too few bytes means no split-K).
cudaError_t oz_product(const OzOperand& a, int64_t a_row0, const OzOperand& b, int64_t b_row0, int64_t M, int64_t N,
                       double alpha, double beta, double* C, int64_t ldc, double* P, size_t p_bytes, int sms,
                       int* status, cudaStream_t st);
// Needs M >= 16, N >= 4, K >= 1; `work` holds oz_work_bytes(M, N, K) bytes
// (digits, exponents and the FP64 split-K partials).
cudaError_t oz_gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work, size_t work_bytes,
                    int sms, int* status, cudaStream_t st);
cudaError_t set_eye_rect(double* X, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st);

}  // namespace rutv
