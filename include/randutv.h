/*
 * randutv.h -- C ABI of the GB300 (sm_103a) randUTV library, librandutv.so.
 *
 * randUTV computes a rank-revealing UTV factorization A = U T V^T of an m x n
 * real matrix (Sec. 1.1, Eq. (1); Sec. 3.1, Eq. (2)): T is upper triangular, U
 * (m x m) and V (n x n) are orthogonal, and the diagonal of T tracks the
 * singular values of A.  It runs the blocked algorithm of Sec. 3.2: for every
 * block of b columns it draws a Gaussian sketch and applies q steps of power
 * iteration (Sec. 3.2.1), builds V_alpha from the Householder QR of the sketch
 * and applies it from the right (compact WY form, Sec. 2.3), builds U_alpha
 * from the Householder QR of the panel and applies it from the left
 * (Sec. 3.2.2), and diagonalises the b x b block with an SVD (Sec. 3.2.3).
 *
 * Conventions shared by every entry point:
 *  - Matrices are FP64, column-major, with the stated leading dimensions.
 *  - Unless an entry point says otherwise, every matrix pointer is a DEVICE
 *    pointer owned by the caller; the library never frees caller memory.
 *  - m >= n >= 0 is required (T upper triangular, Sec. 3.1); b >= 1; q >= 0.
 *  - U == NULL or V == NULL selects the "no orthonormal matrices" mode of
 *    Sec. 6 (T only, or T plus one factor); the work for the missing factor
 *    is skipped.  U and V are accumulated after the last block step from the
 *    reflectors each step keeps (backward order, as LAPACK's dorgqr), which
 *    gives the same factors as updating them at every step, up to rounding.
 *  - T may alias A when lda == m.
 *  - The Gaussian matrix of block step i is G(r, c) = Box-Muller of
 *    Philox4x64-10(counter = (r/4, c, i, 0), key = (seed, 0)), so results are
 *    a deterministic function of (A, b, q, seed, precision); no atomics take
 *    part in any floating-point sum.
 *  - Concurrent calls on one device (several host threads, several streams)
 *    need distinct workspaces; the cached workspace (workspace == NULL) and
 *    the host entry point's cached buffers are shared per device.  Each call
 *    holds a per-device lock while it launches its work, because calls share
 *    the library's side stream; the launched work still overlaps on the GPU.
 *  - Errors detected on the host return at once, before any launch.  Errors
 *    detected on the device (non-finite input, a Jacobi sweep cap, a bounded
 *    wait that ran out) are OR-ed into a device status word and reported
 *    after the stream is synchronised.
 */
#ifndef RANDUTV_H
#define RANDUTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RANDUTV_OK = 0,
    RANDUTV_EINVAL = 1,     /* bad argument (sizes, b, q, leading dimension, NULL T/A) */
    RANDUTV_ENOMEM = 2,     /* device workspace could not be allocated / too small */
    RANDUTV_ENONFINITE = 3, /* a NaN or Inf met in a Householder panel or the SVD */
    RANDUTV_ENOCONV = 4,    /* a b x b Jacobi SVD did not converge within its sweep cap */
    RANDUTV_ETIMEOUT = 5,   /* a bounded inter-block wait gave up (never expected) */
    RANDUTV_ECUDA = 6,      /* a CUDA runtime call failed */
    RANDUTV_ENOTIMPL = 7    /* requested variant is not available */
} randutv_status;

typedef enum {
    RANDUTV_FP64 = 0,               /* every step in FP64 (DMMA tensor cores) */
    RANDUTV_SKETCH_BF16 = 1,        /* sketch and power iteration in BF16 on tcgen05, FP32 accumulate */
    RANDUTV_SKETCH_FP16_SCALED = 2, /* as BF16 with FP16 operands and a per-step scale */
    RANDUTV_SKETCH_FP32 = 3,        /* sketch in FP32 (CUDA cores); used by the batched path */
    RANDUTV_FP64_EMULATED = 4,      /* every FP64 product emulated on BF16 tensor cores (Ozaki scheme,
                                       8 digits of 7 bits, exact FP32 chunks, double-float accumulation);
                                       panels, T factors and the small SVD stay FP64 */
    RANDUTV_EMULATED_SKETCH_BF16 = 5 /* RANDUTV_FP64_EMULATED with the BF16 sketch of RANDUTV_SKETCH_BF16 */
} randutv_precision;

/* Human-readable name of a status code (static string). */
const char* randutv_status_string(int status);

/*
 * randutv_factor -- A = U T V^T by blocked randUTV, FP64 throughout (Sec. 3.2).
 *   m, n     : rows and columns of A, m >= n >= 0.
 *   A        : device, m x n, leading dimension lda >= max(m, 1).  Read only
 *              (unless T aliases it).
 *   b        : block size, b >= 1.  b >= n means a single panel QR + SVD.
 *   q        : power-iteration count, q >= 0 (Sec. 3.2.1).
 *   seed     : key of the counter-based Gaussian generator.
 *   U        : device, m x m, leading dimension m, or NULL.
 *   T        : device, m x n, leading dimension m.  Must not be NULL.
 *   V        : device, n x n, leading dimension n, or NULL.
 * Runs on the legacy default stream, allocates its own workspace (cached per
 * device and reused) and synchronises before returning the status.
 */
randutv_status randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                              uint64_t seed, double* U, double* T, double* V);

/*
 * randutv_factor_ex -- randutv_factor with every option.
 *   prec       : precision variant (randutv_precision): which products run in
 *                FP64, emulated FP64 or a lower precision.  Panel QRs, T factors
 *                and the b x b SVD are FP64 in every variant.
 *   stream     : cudaStream_t to run on (NULL = legacy default stream).
 *   workspace  : device workspace of ws_bytes bytes (see randutv_workspace_size),
 *                or NULL to use the library's cached per-device workspace.
 *   stop_after : stop after this many block steps (< 0: run to completion).  The
 *                partial result is still an exact factorization A = U T V^T whose
 *                leading stop_after*b columns of T are upper triangular (the
 *                early termination of Sec. 1.1 / 3.2).
 *   info       : NULL -> the call synchronises the stream and returns the device
 *                status.  Non-NULL -> DEVICE pointer to one int32 that receives
 *                the device status asynchronously (the call returns RANDUTV_OK
 *                once every launch was queued); read it after synchronising.
 */
randutv_status randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                 uint64_t seed, double* U, double* T, double* V, int prec,
                                 void* stream, void* workspace, size_t ws_bytes, int64_t stop_after,
                                 int* info);

/* Bytes of device workspace randutv_factor_ex needs for these sizes (0 on bad input). */
size_t randutv_workspace_size(int64_t m, int64_t n, int b, int prec);

/*
 * randutv_options -- the variants of randutv_factor_opt, which randutv_factor_ex
 * does not offer.  Initialise with randutv_options_init, then set fields.
 *   prec, stream, workspace, ws_bytes : as randutv_factor_ex (the workspace
 *                size comes from randutv_workspace_size_opt).
 *   stop_after : stop after this many block steps of this call (< 0: none).
 *   rank_tol   : > 0 stops at a tolerance (the early termination at rank k of
 *                Sec. 1.1 and Sec. 3.2, whose cost is O(m n k)): after the
 *                first block step whose smallest diagonal entry satisfies
 *                |T_jj| <= rank_tol * |T_00| (T_00, the largest singular value
 *                estimate, is the first entry of the first block).  The
 *                result is a partial factorization A = U T V^T whose first
 *                cols_done columns of T are upper triangular.  The host reads
 *                each block's diagonal (one synchronisation per block step).
 *   start_col  : > 0 resumes a partial factorization (from stop_after,
 *                rank_tol or an earlier resume): T (m x n) holds it, its
 *                first start_col columns upper triangular, and U, V (when not
 *                NULL) hold its orthogonal factors, which are updated in
 *                place; A is not read (may be NULL).  The block steps
 *                continue with step index start_col / b (start_col must be a
 *                multiple of b, <= n), so the Gaussian draws, and the result,
 *                are those of one uninterrupted call.  Not with qr_first.
 *   qr_first   : 1 = for tall inputs (Sec. 5.1): A = Q_A [R; 0] by blocked
 *                Householder QR (panels of b columns, dlarfg rule, compact WY),
 *                then randUTV of the n x n R = U_R T_R V^T, so that
 *                T = [T_R; 0] and U = Q_A diag(U_R, I).
 *   cols_done  : out: columns of T that are upper triangular on return.
 *   rank       : out: with rank_tol > 0, the number of |T_jj| > rank_tol |T_00|
 *                among those columns; else cols_done.
 */
typedef struct randutv_options {
    int prec;
    void* stream;
    void* workspace;
    size_t ws_bytes;
    int64_t stop_after;
    double rank_tol;
    int64_t start_col;
    int qr_first;
    int64_t cols_done;
    int64_t rank;
} randutv_options;

/* Defaults: RANDUTV_FP64, legacy stream, cached workspace, no stop, no
 * tolerance, start_col 0, qr_first 0. */
void randutv_options_init(randutv_options* opt);

/* Bytes of device workspace randutv_factor_opt needs with these options. */
size_t randutv_workspace_size_opt(int64_t m, int64_t n, int b, const randutv_options* opt);

/*
 * randutv_factor_opt -- randutv_factor_ex with the options above (opt may be
 * NULL for the defaults).  Arguments as randutv_factor; synchronises the
 * stream and returns the status.  RANDUTV_EINVAL also for start_col that is
 * not a multiple of b or exceeds n, start_col with qr_first, or a negative
 * rank_tol.
 */
randutv_status randutv_factor_opt(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                  uint64_t seed, double* U, double* T, double* V, randutv_options* opt);

/*
 * randutv_set_limits -- process-wide limits of the device-side failure
 * detection, for tests of those paths (the paper has no counterpart).
 *   wait_polls : polls after which a grid barrier of the cooperative panel
 *                and Jacobi kernels gives up and the call reports
 *                RANDUTV_ETIMEOUT (each poll sleeps 64-256 ns); <= 0 restores
 *                the default (2^23 polls, about a second).
 *   max_sweeps : sweep cap of every b x b Jacobi SVD, after which the call
 *                reports RANDUTV_ENOCONV; <= 0 restores the default (30).
 * Takes effect for launches made after it returns; not for the batched path.
 */
void randutv_set_limits(int64_t wait_polls, int max_sweeps);

/*
 * randutv_factor_host -- randutv_factor on HOST buffers: copies A to the device,
 * factors it, copies U, T, V back (U or V NULL skips that factor).  A (lda >= m),
 * U (m x m), T (m x n), V (n x n) are host pointers, column-major.  Page-locked
 * (pinned) host buffers are read and written by the library's own copy
 * kernels through their device addresses (these keep the host link's full
 * rate, where DMA copies were measured an order of magnitude slower after
 * the link had been idle); other host memory goes through cudaMemcpy.  The device copies of A/T, U
 * and V live in buffers the library caches per device and grows as needed
 * (like the workspace), so repeated calls do not allocate; calls on one device
 * must therefore not overlap (from several host threads).  Synchronous.
 */
randutv_status randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                   uint64_t seed, double* U, double* T, double* V, int prec);

/*
 * Batched randUTV: `count` independent factorizations (each as randutv_factor,
 * FP64, or with RANDUTV_SKETCH_FP32 for an FP32 sketch) in ONE persistent
 * kernel.  Each CTA of the kernel pops the next matrix from an atomic queue
 * ordered longest-processing-time first and runs every block step of the
 * matrix itself.  Per-matrix block sizes come from an autotune table.
 *   m, n, lda, seed : host arrays of count entries (m[i] >= n[i], m[i] <= 8192).
 *   A, T            : host arrays of count DEVICE pointers (A[i] with ld lda[i],
 *                     T[i] m[i] x n[i] with ld m[i]); U, V: host arrays of device pointers
 *                     (m x m / n x n) or NULL (no orthonormal factors).
 *   q               : power-iteration count for every matrix.
 *   prec            : RANDUTV_FP64 or RANDUTV_SKETCH_FP32.
 *   autotune_table  : text with lines "nmin nmax tall b [tile]" (tall: 1 =
 *                     m > n, 0 = square, -1 = any; tile: the output tile of
 *                     the per-matrix DMMA products, 32 or 64, default 64)
 *                     and an optional line "threads NT" (threads per CTA,
 *                     i.e. per matrix in flight: 128 or 256, default 256),
 *                     e.g. the output of randutv_batched_autotune; NULL =
 *                     built-in table.  Block sizes are clamped to [1, 64].
 *   status          : host array of count statuses (or NULL), filled on return.
 * randutv_batched builds a plan, runs it once and frees it (synchronous).
 * A plan keeps the descriptors on the device and holds the launch as a CUDA
 * graph; randutv_batched_plan_run replays it (synchronous; the matrices the
 * pointers name are re-factored from A each run).
 */
typedef struct randutv_batch_plan randutv_batch_plan;

randutv_status randutv_batched(int count, const int64_t* m, const int64_t* n, const double* const* A,
                               const int64_t* lda, double* const* U, double* const* T, double* const* V,
                               const uint64_t* seed, int q, int prec, const char* autotune_table, int* status,
                               void* stream);
randutv_status randutv_batched_plan_create(int count, const int64_t* m, const int64_t* n, const double* const* A,
                                           const int64_t* lda, double* const* U, double* const* T, double* const* V,
                                           const uint64_t* seed, int q, int prec, const char* autotune_table,
                                           randutv_batch_plan** plan);
randutv_status randutv_batched_plan_run(randutv_batch_plan* plan, int* status, void* stream);
void randutv_batched_plan_destroy(randutv_batch_plan* plan);

/*
 * randutv_batched_autotune: for each size class (n in [2^k, 2^(k+1)), square
 * and tall separately) times the batched kernel on up to 608 members of the
 * class with b = 16, 32, 64 and GEMM tiles of 32 and 64, keeps the fastest,
 * then times the whole batch with 128 and 256 threads per matrix, and writes
 * the result as a table (the format randutv_batched reads) into table_out
 * (host, table_bytes bytes).  Overwrites T, U, V of the matrices it runs.
 * Synchronous.
 */
randutv_status randutv_batched_autotune(int count, const int64_t* m, const int64_t* n, const double* const* A,
                                        const int64_t* lda, double* const* U, double* const* T, double* const* V,
                                        const uint64_t* seed, int q, int prec, char* table_out, size_t table_bytes,
                                        void* stream);

/*
 * Learned power-iteration count.  Sec. 3.2.1 uses a fixed q; here, before the
 * sketch of every block step, a small network (16 -> 64 -> 64 -> 4, GELU,
 * FP32, softmax over q in {0,1,2,3}) picks q from 16 features: the decay of
 * the previous block's panel-QR R diagonal and of the Householder R diagonal of the
 * q = 0 sketch (compressed to 2b rows by a CountSketch with random signs),
 * each as log10(|d_j| / |d_0|) at j = w/8, ..., 7w/8, and the level of the
 * trailing matrix, log10 of the compressed sketch's Frobenius norm over the
 * first block's (it tells a block of rounding noise from a cluster).
 * The q = 0 product is reused by the chosen iterations.
 *   model   : HOST array of randutv_learnq_model_floats() floats (layout:
 *             W1[16][64] b1[64] W2[64][64] b2[64] W3[64][4] b3[4] mu[16] sd[16],
 *             inputs standardised as (f - mu) / sd), or NULL -> fixed q = 2.
 *             A non-finite network output also falls back to q = 2.  The
 *             network predicts a distribution over the smallest adequate q;
 *             the step runs the smallest q whose cumulative predicted
 *             probability reaches 0.999.
 *   q_used  : HOST array of ceil(n / b) ints (or NULL): the q chosen per
 *             sketch step, -1 for the final block (no sketch).
 * Other arguments as randutv_factor / randutv_factor_ex.  The choice stays
 * on the device: every power iteration up to q = 3 is queued, and its
 * kernels return at once when the chosen q is smaller, so the host never
 * waits for a block step; q_used is filled once, when the call ends.  Each
 * block's b x b SVD overlaps the next step on a side stream, as in the
 * fixed-q path (the features need only the previous panel's R diagonal).
 */
int randutv_learnq_model_floats(void);
randutv_status randutv_factor_learnedq(int64_t m, int64_t n, const double* A, int64_t lda, int b,
                                       const float* model, uint64_t seed, double* U, double* T, double* V,
                                       int* q_used);
randutv_status randutv_factor_learnedq_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b,
                                          const float* model, uint64_t seed, double* U, double* T, double* V,
                                          int* q_used, int prec, void* stream);

/*
 * Training data for the network, generated by the method itself: factors A
 * (device, T device m x n, U and V not formed) along the q = 2 trajectory and,
 * for each sketch step (up to max_blocks), writes the 16 features (HOST
 * float[16] each), the label (HOST int: the smallest q in {0,1,2} whose
 * diagonal sigma(T22 Q1(q)) stays within 5% of the q = 2 one, entry by entry),
 * and optionally the four candidate diagonals (HOST double[4 * b] each).
 * Diagonal entries below 1e-13 times the first block's largest are rounding
 * noise and take no part in the label.
 * *nblocks receives the number of steps written.
 */
randutv_status randutv_learnq_trace(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                                    double* T, float* features, int* labels, double* candidates,
                                    int64_t max_blocks, int64_t* nblocks);
/* As randutv_learnq_trace, with the products in `prec` (RANDUTV_FP64 or
 * RANDUTV_FP64_EMULATED) and only every stride-th sketch step recorded (step
 * 0 and the steps i with i % stride == seed % stride; the others run the q = 2
 * step alone), which makes traces of many large matrices affordable.
 * stride >= 1.  Labels skip diagonal entries below 1e-13 times the first
 * block's largest (rounding noise); a block of noise alone is labelled 0. */
randutv_status randutv_learnq_trace_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                                       double* T, float* features, int* labels, double* candidates,
                                       int64_t max_blocks, int64_t* nblocks, int prec, int64_t stride);

/*
 * Network training and evaluation on the GPU with the library's own kernels
 * (all host arrays; the library allocates and frees its device copies):
 *   randutv_learnq_train   : `epochs` full-batch Adam steps (lr, weight decay
 *                            wd) on the mean cross-entropy of X (N x 16,
 *                            row-major) against labels y; model in/out;
 *                            loss_history (epochs floats) or NULL.
 *   randutv_learnq_grad    : gradient of that loss at `model` (grad has the
 *                            model's length; mu and sd entries are left 0)
 *                            and the loss itself.
 *   randutv_learnq_predict : softmax probabilities (N x 4) of the network.
 */
randutv_status randutv_learnq_train(const float* X, const int* y, int N, int epochs, float lr, float wd,
                                    float* model, float* loss_history);
randutv_status randutv_learnq_grad(const float* X, const int* y, int N, const float* model, float* grad,
                                   float* loss);
randutv_status randutv_learnq_predict(const float* model, const float* X, int N, float* probs);

/*
 * randutv_svd_small_noalloc -- the b x b SVD step (one-sided Jacobi, the
 * kernel randutv_factor runs on every diagonal block) for callers that cannot
 * allocate device memory: code under an allocator that forbids cudaMalloc,
 * allocation-free real-time paths, or plugins whose host framework owns all
 * device memory.  The paper has no counterpart; it is a packaging of an
 * existing kernel.
 *   w          : order of R, 0 <= w <= RANDUTV_SVD_NOALLOC_MAX_W (larger w
 *                returns RANDUTV_EINVAL).
 *   R          : device, w x w, leading dimension ldr >= w; only its upper
 *                triangle is read.
 *   D, Us, Vs  : device outputs: D (w) descending singular values, Us and Vs
 *                (w x w, ld w) with R = Us diag(D) Vs^T, each pair signed so
 *                that the largest entry of Vs(:, j) is positive.
 *   stream     : cudaStream_t (NULL = legacy default stream).  Synchronous.
 * The scratch (the Jacobi working copies, barrier and status words) is a
 * fixed device array inside the library, about 1 MiB, that every GPU which
 * loads the library holds until the process exits; no call allocates or
 * frees memory.  The first call on a device looks up that array's device
 * address, so make it before any CUDA stream capture.  All calls on a device
 * share the array: calls that overlap on the GPU (other host threads, other
 * streams) race and must be serialised by the caller.
 */
#define RANDUTV_SVD_NOALLOC_MAX_W 256
randutv_status randutv_svd_small_noalloc(int w, const double* R, int64_t ldr, double* D, double* Us, double* Vs,
                                         void* stream);

/*
 * Tracing (the per-task time breakdown of Sec. 5.4 / Sec. 6.1, done with CUDA
 * events).  While enabled, every launcher of the library brackets its kernel
 * launches with a pair of CUDA events on its stream and records the
 * algorithmic flops and bytes of the launch under a class name.
 *   randutv_trace_enable(on)  : 1 = start recording, 0 = stop; returns the
 *                               previous setting.
 *   randutv_trace_read(out,n) : synchronises the recorded events and writes up
 *                               to n per-class totals into out (host array);
 *                               returns the number of classes.
 *   randutv_trace_reset()     : drops all records.
 *   randutv_launch_count()    : kernels launched by this library since load.
 */
typedef struct randutv_trace_class {
    char name[32];      /* kernel class, e.g. "gemm_right" */
    int64_t scopes;     /* launcher calls */
    int64_t kernels;    /* kernel launches inside them */
    double ms;          /* summed event time */
    double flops;       /* summed algorithmic flops */
    double bytes;       /* summed algorithmic bytes */
} randutv_trace_class;

int randutv_trace_enable(int on);
int randutv_trace_read(randutv_trace_class* out, int max_classes);
void randutv_trace_reset(void);
long long randutv_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* RANDUTV_H */
