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
 *    is skipped.
 *  - T may alias A when lda == m.
 *  - The Gaussian matrix of block step i is G(r, c) = Box-Muller of
 *    Philox4x64-10(counter = (r/4, c, i, 0), key = (seed, 0)), so results are
 *    a deterministic function of (A, b, q, seed, precision); no atomics take
 *    part in any floating-point sum.
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
    RANDUTV_SKETCH_FP32 = 3         /* sketch in FP32 (CUDA cores); used by the batched path */
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
 *   prec       : precision of the sketch (randutv_precision); everything else is FP64.
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
 * randutv_factor_host -- randutv_factor on HOST buffers: copies A to the device,
 * factors it, copies U, T, V back (U or V NULL skips that factor).  Allocates
 * and frees its own device buffers.  A (lda >= m), U (m x m), T (m x n),
 * V (n x n) are host pointers, column-major.  Synchronous.
 */
randutv_status randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                   uint64_t seed, double* U, double* T, double* V, int prec);

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
typedef struct {
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
