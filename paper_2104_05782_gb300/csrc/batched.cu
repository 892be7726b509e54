// batched.cu -- many independent randUTV factorizations in one persistent launch.
//
// Thousands of small matrices (n in [32, 512]) leave a per-matrix launch
// sequence (tens of kernels per block step) launch bound, and one matrix is
// far too small to fill 152 SMs.  Here each CTA is a complete randUTV
// engine: it pops the next matrix from an atomic queue (the host orders the
// queue longest-processing-time first, which bounds the makespan), and runs
// every part of the block step of Sec. 3.2 on it with CTA-level device
// functions -- DMMA (mma.sync f64) GEMM tiles for the sketch, the WY updates
// (Sec. 2.3) and the small-SVD application, a Householder panel with the
// dlarfg rule, the compact-WY triangular factor, and a one-sided Jacobi SVD
// held in shared memory -- with the same conventions as the single-matrix
// path (Gaussian draw, signs, ordering), so each matrix matches the oracle.
// Nothing waits on another CTA: the queue pop is one atomicAdd.
//
// Tunable shape: the engine is compiled for 128 and 256 threads per CTA
// (threads per matrix in flight, one choice per plan), and its DMMA GEMM for
// 32 x 32 and 64 x 64 output tiles (chosen per matrix); with the block size
// b per size class, randutv_batched_autotune times these choices.
//
// The optional FP32 sketch (RANDUTV_SKETCH_FP32) runs the sketch products on
// the FP32 pipe (about 70x the FP64 rate on GB300) with an FP32 classical
// Gram-Schmidt (twice) re-orthonormalisation between products; the rest is FP64.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/randutv.h"
#include "common.cuh"
#include "internal.h"
#include "philox.cuh"
#include "trace.h"

namespace rutv {

namespace {

constexpr int kMaxThreads = 256;  // threads per CTA: 128 or 256 (the template parameter NT)
constexpr int kMaxWarps = kMaxThreads / 32;
constexpr int BMAX = 64;  // largest block size of the batched path
constexpr int kBatchedMaxSweeps = 30;

struct BatchDesc {
    int64_t m, n, lda;
    const double* A;
    double *U, *T, *V;
    uint64_t seed;
    int b, status;
    int tile;  // GEMM tile of this matrix (32 or 64)
};

struct Slot {  // per-CTA workspace, sized for the largest matrix of the batch
    double *G, *Y, *Z, *W, *X, *X2, *tmp, *tau, *Tf, *gram, *D, *Us, *Vs;
    float *Yf, *Zf;
};

struct BSmem {
    double As[16][64 + 2];
    double Bs[16][64 + 2];
    double red[kMaxWarps * 3];
    double wv[BMAX + 2];
    double sc[4];
    double jA[BMAX * BMAX];
    double jV[BMAX * BMAX];
    int flag;
};

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

// C = alpha op(A) op(B) + beta C over the whole CTA of NT threads (128 or
// 256), TILE x TILE output tiles (32 or 64), 16-deep k steps staged in shared
// memory.  The warps form a 2 x (NT / 64) grid, each owning a
// (TILE / 2) x (2 TILE / (NT / 32)) block of m8n8k4 DMMA fragments.
template <bool TA, bool TB, int TILE, int NT>
__device__ void cta_gemm(int M, int N, int K, double alpha, const double* A, int64_t lda, const double* B,
                         int64_t ldb, double beta, double* C, int64_t ldc, BSmem& sm) {
    constexpr int BNW = NT / 32;
    constexpr int WR = TILE / 2, WC = 2 * TILE / BNW, FI = WR / 8, FJ = WC / 8;
    constexpr int LOADS = TILE * 16 / NT;  // elements of each operand tile per thread and k step
    static_assert(FI >= 1 && FJ >= 1 && LOADS >= 1, "tile and thread count");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 1) * WR, wn = (warp >> 1) * WC;
    const int tm = (M + TILE - 1) / TILE, tn = (N + TILE - 1) / TILE;
    for (int t = 0; t < tm * tn; ++t) {
        const int row0 = (t % tm) * TILE, col0 = (t / tm) * TILE;
        double acc[FI][FJ][2];
#pragma unroll
        for (int i = 0; i < FI; ++i)
#pragma unroll
            for (int j = 0; j < FJ; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
        for (int k0 = 0; k0 < K; k0 += 16) {
            __syncthreads();
#pragma unroll
            for (int it = 0; it < LOADS; ++it) {
                int idx = tid + it * NT;
                int m, k;
                if (!TA) { m = idx % TILE; k = idx / TILE; } else { k = idx % 16; m = idx / 16; }
                int gi = row0 + m, gk = k0 + k;
                double v = 0.0;
                if (gi < M && gk < K) v = TA ? A[gk + (int64_t)gi * lda] : A[gi + (int64_t)gk * lda];
                sm.As[k][m] = v;
                int n, kk;
                if (TB) { n = idx % TILE; kk = idx / TILE; } else { kk = idx % 16; n = idx / 16; }
                int gj = col0 + n, gk2 = k0 + kk;
                double u = 0.0;
                if (gj < N && gk2 < K) u = TB ? B[gj + (int64_t)gk2 * ldb] : B[gk2 + (int64_t)gj * ldb];
                sm.Bs[kk][n] = u;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; kk += 4) {
                double af[FI], bf[FJ];
#pragma unroll
                for (int i = 0; i < FI; ++i) af[i] = sm.As[kk + (lane & 3)][wm + i * 8 + (lane >> 2)];
#pragma unroll
                for (int j = 0; j < FJ; ++j) bf[j] = sm.Bs[kk + (lane & 3)][wn + j * 8 + (lane >> 2)];
#pragma unroll
                for (int i = 0; i < FI; ++i)
#pragma unroll
                    for (int j = 0; j < FJ; ++j) dmma(acc[i][j], af[i], bf[j]);
            }
        }
#pragma unroll
        for (int i = 0; i < FI; ++i) {
            int gi = row0 + wm + i * 8 + (lane >> 2);
            if (gi >= M) continue;
#pragma unroll
            for (int j = 0; j < FJ; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int gj = col0 + wn + j * 8 + 2 * (lane & 3) + h;
                    if (gj >= N) continue;
                    double* c = C + gi + (int64_t)gj * ldc;
                    double v = alpha * acc[i][j][h];
                    *c = (beta == 0.0) ? v : v + beta * (*c);
                }
        }
    }
    __syncthreads();
}

template <int NT, int TILE>
__device__ void cta_gemm_t(bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int64_t lda,
                           const double* B, int64_t ldb, double beta, double* C, int64_t ldc, BSmem& sm) {
    if (!ta && !tb) cta_gemm<false, false, TILE, NT>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
    else if (ta && !tb) cta_gemm<true, false, TILE, NT>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
    else if (!ta && tb) cta_gemm<false, true, TILE, NT>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
    else cta_gemm<true, true, TILE, NT>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
}

// tile: the matrix's GEMM tile (32 or 64), chosen per matrix by the autotune table
template <int NT>
__device__ void cta_gemm_dispatch(int tile, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                                  int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                                  BSmem& sm) {
    if (M <= 0 || N <= 0) return;
    if (tile == 32) cta_gemm_t<NT, 32>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
    else cta_gemm_t<NT, 64>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
}

template <int NT>
__device__ double block_sum(double v, BSmem& sm) {
    constexpr int BNW = NT / 32;
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < BNW; ++k) s += sm.red[k];
    return s;
}

// Householder QR of P (len x w, ld), dlarfg rule (as the panel kernel).
template <int NT>
__device__ void cta_householder(double* P, int64_t ld, int len, int w, double* tau, int* status, BSmem& sm) {
    constexpr int BNT = NT, BNW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < w && j < len; ++j) {
        double s = 0.0;
        for (int r = j + 1 + tid; r < len; r += BNT) {
            double x = P[r + (int64_t)j * ld];
            s += x * x;
        }
        const double xi2 = block_sum<NT>(s, sm);
        const double alpha = P[j + (int64_t)j * ld];
        double tj = 0.0, beta = alpha, d = 1.0;
        bool act = false;
        if (!isfinite(xi2) || !isfinite(alpha)) {
            if (tid == 0) atomicOr(status, ST_NONFINITE);
        } else if (xi2 > 0.0) {
            double h = hypot(alpha, sqrt(xi2));
            beta = (alpha >= 0.0) ? -h : h;
            tj = (beta - alpha) / beta;
            d = alpha - beta;
            act = true;
        }
        __syncthreads();
        if (tid == 0) tau[j] = tj;
        if (!act) continue;
        for (int r = j + 1 + tid; r < len; r += BNT) P[r + (int64_t)j * ld] /= d;
        __syncthreads();
        if (tid == 0) P[j + (int64_t)j * ld] = beta;
        for (int c = j + 1 + warp; c < w; c += BNW) {
            double acc = 0.0;
            for (int r = j + 1 + lane; r < len; r += 32) acc += P[r + (int64_t)j * ld] * P[r + (int64_t)c * ld];
            acc = warp_sum(acc);
            if (lane == 0) sm.wv[c] = P[j + (int64_t)c * ld] + acc;
        }
        __syncthreads();
        const int rows = len - j, cols = w - j - 1;
        for (int e = tid; e < rows * cols; e += BNT) {
            int r = j + e % rows, c = j + 1 + e / rows;
            double v = (r == j) ? 1.0 : P[r + (int64_t)j * ld];
            P[r + (int64_t)c * ld] -= tj * v * sm.wv[c];
        }
        __syncthreads();
    }
    __syncthreads();
}

template <int NT>
__device__ void cta_extract_w(const double* P, int64_t ld, int len, int w, double* W) {
    constexpr int BNT = NT;
    for (int e = threadIdx.x; e < len * w; e += BNT) {
        int r = e % len, c = e / len;
        W[e] = (r < c) ? 0.0 : (r == c ? 1.0 : P[r + (int64_t)c * ld]);
    }
    __syncthreads();
}

// Tf(j,j) = tau_j, Tf(0:j, j) = -tau_j Tf(0:j,0:j) gram(0:j, j)  (Sec. 2.3)
template <int NT>
__device__ void cta_tfactor(const double* gram, const double* tau, int w, double* Tf) {
    constexpr int BNT = NT, BNW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < w * w; e += BNT) Tf[e] = 0.0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        const double tj = tau[j];
        for (int i = warp; i < j; i += BNW) {
            double s = 0.0;
            for (int l = i + lane; l < j; l += 32) s += Tf[i + (int64_t)l * w] * gram[l + (int64_t)j * w];
            s = warp_sum(s);
            if (lane == 0) Tf[i + (int64_t)j * w] = -tj * s;
        }
        if (tid == 0) Tf[j + (int64_t)j * w] = tj;
        __syncthreads();
    }
}

// One-sided Jacobi SVD of the upper triangle of R (w x w, w <= BMAX) in shared
// memory; circle ordering, one warp per pair; canonical output as svd.cu.
template <int NT>
__device__ void cta_jacobi(const double* R, int64_t ldr, int w, double* D, double* Us, double* Vs, int* status,
                           BSmem& sm) {
    constexpr int BNT = NT, BNW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* A = sm.jA;
    double* V = sm.jV;
    for (int e = tid; e < w * w; e += BNT) {
        int r = e % w, c = e / w;
        A[e] = (r <= c) ? R[r + (int64_t)c * ldr] : 0.0;
        V[e] = (r == c) ? 1.0 : 0.0;
    }
    const int n2 = w + (w & 1);
    const double tol = (double)w * 1.1102230246251565e-16;
    bool converged = (w <= 1);
    for (int sweep = 0; sweep < kBatchedMaxSweeps && !converged; ++sweep) {
        __syncthreads();
        if (tid == 0) sm.flag = 0;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            for (int k = warp; k < n2 / 2; k += BNW) {
                int p = (k == 0) ? 0 : 1 + (k - 1 + round) % (n2 - 1);
                int kq = n2 - 1 - k;
                int q = (kq == 0) ? 0 : 1 + (kq - 1 + round) % (n2 - 1);
                if (p > q) { int t = p; p = q; q = t; }
                if (q >= w) continue;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < w; r += 32) {
                    double x = A[r + p * w], y = A[r + q * w];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (!isfinite(al) || !isfinite(be) || !isfinite(ga)) {
                    if (lane == 0) atomicOr(status, ST_NONFINITE);
                    continue;
                }
                if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t);
                double sn = cs * t;
                for (int r = lane; r < w; r += 32) {
                    double x = A[r + p * w], y = A[r + q * w];
                    A[r + p * w] = cs * x - sn * y;
                    A[r + q * w] = sn * x + cs * y;
                    double u = V[r + p * w], z = V[r + q * w];
                    V[r + p * w] = cs * u - sn * z;
                    V[r + q * w] = sn * u + cs * z;
                }
                if (lane == 0) sm.flag = 1;
            }
            __syncthreads();
        }
        converged = (sm.flag == 0);
    }
    __syncthreads();
    if (!converged && tid == 0) atomicOr(status, ST_NOCONV);
    double* nrm = sm.wv;
    for (int c = tid; c < w; c += BNT) {
        double s = 0.0;
        for (int r = 0; r < w; ++r) s += A[r + c * w] * A[r + c * w];
        nrm[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < w; c += BNT) {
        double v = nrm[c];
        int rank = 0;
        for (int c2 = 0; c2 < w; ++c2) rank += (nrm[c2] > v) || (nrm[c2] == v && c2 < c);
        D[rank] = v;
        for (int r = 0; r < w; ++r) {
            Vs[r + (int64_t)rank * w] = V[r + c * w];
            Us[r + (int64_t)rank * w] = (v > 0.0) ? A[r + c * w] / v : 0.0;
        }
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < w; ++j) {
            if (D[j] > 0.0) continue;
            for (int e = 0; e < w; ++e) {
                double* u = Us + (int64_t)j * w;
                for (int r = 0; r < w; ++r) u[r] = (r == e) ? 1.0 : 0.0;
                for (int pass = 0; pass < 2; ++pass)
                    for (int l = 0; l < w; ++l) {
                        if (l == j || (D[l] == 0.0 && l > j)) continue;
                        const double* ul = Us + (int64_t)l * w;
                        double d = 0.0;
                        for (int r = 0; r < w; ++r) d += ul[r] * u[r];
                        for (int r = 0; r < w; ++r) u[r] -= d * ul[r];
                    }
                double nn = 0.0;
                for (int r = 0; r < w; ++r) nn += u[r] * u[r];
                nn = sqrt(nn);
                if (nn > 0.5) {
                    for (int r = 0; r < w; ++r) u[r] /= nn;
                    break;
                }
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < w; j += BNT) {
        int imax = 0;
        double vmax = -1.0;
        for (int r = 0; r < w; ++r) {
            double a = fabs(Vs[r + (int64_t)j * w]);
            if (a > vmax) { vmax = a; imax = r; }
        }
        if (Vs[imax + (int64_t)j * w] < 0.0)
            for (int r = 0; r < w; ++r) {
                Vs[r + (int64_t)j * w] = -Vs[r + (int64_t)j * w];
                Us[r + (int64_t)j * w] = -Us[r + (int64_t)j * w];
            }
    }
    __syncthreads();
}

template <int NT>
__device__ void cta_copy(const double* src, int64_t lds, double* dst, int64_t ldd, int rows, int cols) {
    constexpr int BNT = NT;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += BNT) {
        int64_t i = e % rows, j = e / rows;
        dst[i + j * ldd] = src[i + j * lds];
    }
    __syncthreads();
}

struct MatCtx {
    int64_t m, n;
    int b, q, prec, tile;
    uint64_t seed;
    double *U, *T, *V;
    Slot s;
    int* status;
};

template <int NT>
__device__ void b_factor_panel(MatCtx& c, double* P, int64_t ld, int len, int w, BSmem& sm) {
    cta_householder<NT>(P, ld, len, w, c.s.tau, c.status, sm);
    cta_extract_w<NT>(P, ld, len, w, c.s.W);
    cta_gemm_dispatch<NT>(c.tile, true, false, w, w, len, 1.0, c.s.W, len, c.s.W, len, 0.0, c.s.gram, w, sm);
    cta_tfactor<NT>(c.s.gram, c.s.tau, w, c.s.Tf);
}

template <int NT>
__device__ void b_apply_right(MatCtx& c, double* C, int64_t ldc, int rows, int cols, int w, BSmem& sm) {
    if (rows <= 0 || cols <= 0) return;
    cta_gemm_dispatch<NT>(c.tile, false, false, rows, w, cols, 1.0, C, ldc, c.s.W, cols, 0.0, c.s.X, rows, sm);
    cta_gemm_dispatch<NT>(c.tile, false, false, rows, w, w, 1.0, c.s.X, rows, c.s.Tf, w, 0.0, c.s.X2, rows, sm);
    cta_gemm_dispatch<NT>(c.tile, false, true, rows, cols, w, -1.0, c.s.X2, rows, c.s.W, cols, 1.0, C, ldc, sm);
}

template <int NT>
__device__ void b_apply_left_t(MatCtx& c, double* C, int64_t ldc, int len, int cols, int w, BSmem& sm) {
    if (len <= 0 || cols <= 0) return;
    cta_gemm_dispatch<NT>(c.tile, true, false, w, cols, len, 1.0, c.s.W, len, C, ldc, 0.0, c.s.X, w, sm);
    cta_gemm_dispatch<NT>(c.tile, true, false, w, cols, w, 1.0, c.s.Tf, w, c.s.X, w, 0.0, c.s.X2, w, sm);
    cta_gemm_dispatch<NT>(c.tile, false, false, len, cols, w, -1.0, c.s.W, len, c.s.X2, w, 1.0, C, ldc, sm);
}

template <int NT>
__device__ void b_panel_and_svd(MatCtx& c, int64_t k0, int w, BSmem& sm) {
    constexpr int BNT = NT;
    const int m = (int)c.m, n = (int)c.n;
    const int mp = m - (int)k0;
    double* T = c.T;
    double* P = T + k0 + k0 * m;
    b_factor_panel<NT>(c, P, m, mp, w, sm);
    b_apply_left_t<NT>(c, T + k0 + (k0 + w) * m, m, mp, n - (int)k0 - w, w, sm);
    if (c.U) b_apply_right<NT>(c, c.U + k0 * m, m, m, mp, w, sm);
    cta_jacobi<NT>(P, m, w, c.s.D, c.s.Us, c.s.Vs, c.status, sm);
    if (k0 > 0) {
        cta_gemm_dispatch<NT>(c.tile, false, false, (int)k0, w, w, 1.0, T + k0 * m, m, c.s.Vs, w, 0.0, c.s.tmp, k0, sm);
        cta_copy<NT>(c.s.tmp, k0, T + k0 * m, m, (int)k0, w);
    }
    const int nr = n - (int)k0 - w;
    if (nr > 0) {
        cta_gemm_dispatch<NT>(c.tile, true, false, w, nr, w, 1.0, c.s.Us, w, T + k0 + (k0 + w) * m, m, 0.0, c.s.tmp, w, sm);
        cta_copy<NT>(c.s.tmp, w, T + k0 + (k0 + w) * m, m, w, nr);
    }
    for (int64_t e = threadIdx.x; e < (int64_t)mp * w; e += BNT) {
        int64_t i = e % mp, j = e / mp;
        T[(k0 + i) + (k0 + j) * m] = (i == j) ? c.s.D[j] : 0.0;
    }
    __syncthreads();
    if (c.V) {
        cta_gemm_dispatch<NT>(c.tile, false, false, n, w, w, 1.0, c.V + k0 * n, n, c.s.Vs, w, 0.0, c.s.tmp, n, sm);
        cta_copy<NT>(c.s.tmp, n, c.V + k0 * n, n, n, w);
    }
    if (c.U) {
        cta_gemm_dispatch<NT>(c.tile, false, false, m, w, w, 1.0, c.U + k0 * m, m, c.s.Us, w, 0.0, c.s.tmp, m, sm);
        cta_copy<NT>(c.s.tmp, m, c.U + k0 * m, m, m, w);
    }
}

// FP32 sketch product on CUDA cores: Out (M x b, FP32) = op(T22) In (K x b),
// op = transpose (Y = T22^T In) or not (Z = T22 In).  T22 read in FP64.
template <int NT>
__device__ void cta_sgemm_sketch(bool trans, int M, int K, int b, const double* T22, int64_t ldt, const float* In,
                                 float* Out) {
    constexpr int BNT = NT;
    for (int e = threadIdx.x; e < M * b; e += BNT) {
        int i = e % M, j = e / M;
        float s = 0.0f;
        const float* x = In + (int64_t)j * K;
        if (trans)
            for (int k = 0; k < K; ++k) s = fmaf((float)T22[k + (int64_t)i * ldt], x[k], s);
        else
            for (int k = 0; k < K; ++k) s = fmaf((float)T22[i + (int64_t)k * ldt], x[k], s);
        Out[i + (int64_t)j * M] = s;
    }
    __syncthreads();
}

// FP32 classical Gram-Schmidt with reorthogonalisation (CGS2) on the columns
// of X (L x b): for each column, two passes of h = X(:,0:j)^T x_j,
// x_j -= X(:,0:j) h, then normalisation.
template <int NT>
__device__ void cta_cgs2_32(float* X, int L, int b, BSmem& sm) {
    constexpr int BNT = NT, BNW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < b; ++j) {
        float* xj = X + (int64_t)j * L;
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            for (int i = warp; i < j; i += BNW) {
                const float* xi = X + (int64_t)i * L;
                float d = 0.0f;
                for (int r = lane; r < L; r += 32) d = fmaf(xi[r], xj[r], d);
                d = warp_sum_f(d);
                if (lane == 0) sm.wv[i] = (double)d;
            }
            __syncthreads();
            for (int r = tid; r < L; r += BNT) {
                float s = 0.0f;
                for (int i = 0; i < j; ++i) s = fmaf((float)sm.wv[i], X[r + (int64_t)i * L], s);
                xj[r] -= s;
            }
            __syncthreads();
        }
        float nn = 0.0f;
        for (int r = tid; r < L; r += BNT) nn = fmaf(xj[r], xj[r], nn);
        const double tot = block_sum<NT>((double)nn, sm);
        const float inv = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.0f;
        for (int r = tid; r < L; r += BNT) xj[r] *= inv;
        __syncthreads();
    }
}

template <int NT>
__device__ void b_sketch_step(MatCtx& c, int64_t i, BSmem& sm) {
    constexpr int BNT = NT;
    const int m = (int)c.m, n = (int)c.n, b = c.b;
    const int64_t k0 = i * (int64_t)b;
    const int mp = m - (int)k0, np = n - (int)k0;
    double* T22 = c.T + k0 + k0 * m;
    // Gaussian G^(i) (m' x b)
    const int groups = (mp + 3) / 4;
    for (int e = threadIdx.x; e < groups * b; e += BNT) {
        int k = e % groups, col = e / groups;
        double z[4];
        gaussian4(c.seed, i, k, col, z);
        for (int t = 0; t < 4; ++t) {
            int r = 4 * k + t;
            if (r < mp) c.s.G[r + (int64_t)col * mp] = z[t];
        }
    }
    __syncthreads();
    if (c.prec == RANDUTV_SKETCH_FP32) {
        float* Gf = c.s.Zf;
        for (int e = threadIdx.x; e < mp * b; e += BNT) Gf[e] = (float)c.s.G[e];
        __syncthreads();
        cta_sgemm_sketch<NT>(true, np, mp, b, T22, m, Gf, c.s.Yf);
        for (int it = 0; it < c.q; ++it) {
            cta_cgs2_32<NT>(c.s.Yf, np, b, sm);
            cta_sgemm_sketch<NT>(false, mp, np, b, T22, m, c.s.Yf, c.s.Zf);
            cta_cgs2_32<NT>(c.s.Zf, mp, b, sm);
            cta_sgemm_sketch<NT>(true, np, mp, b, T22, m, c.s.Zf, c.s.Yf);
        }
        for (int e = threadIdx.x; e < np * b; e += BNT) c.s.Y[e] = (double)c.s.Yf[e];
        __syncthreads();
    } else {
        cta_gemm_dispatch<NT>(c.tile, true, false, np, b, mp, 1.0, T22, m, c.s.G, mp, 0.0, c.s.Y, np, sm);
        for (int it = 0; it < c.q; ++it) {
            cta_gemm_dispatch<NT>(c.tile, false, false, mp, b, np, 1.0, T22, m, c.s.Y, np, 0.0, c.s.Z, mp, sm);
            cta_gemm_dispatch<NT>(c.tile, true, false, np, b, mp, 1.0, T22, m, c.s.Z, mp, 0.0, c.s.Y, np, sm);
        }
    }
    b_factor_panel<NT>(c, c.s.Y, np, np, b, sm);
    b_apply_right<NT>(c, c.T + k0 * m, m, m, np, b, sm);
    if (c.V) b_apply_right<NT>(c, c.V + k0 * n, n, n, np, b, sm);
    b_panel_and_svd<NT>(c, k0, b, sm);
}

template <int NT>
__device__ void b_factor_one(MatCtx& c, const double* A, int64_t lda, BSmem& sm) {
    constexpr int BNT = NT;
    const int m = (int)c.m, n = (int)c.n;
    for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += BNT) {
        int64_t i = e % m, j = e / m;
        double v = A[i + j * lda];
        if (!isfinite(v)) atomicOr(c.status, ST_NONFINITE);
        c.T[i + j * m] = v;
    }
    if (c.U)
        for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += BNT) c.U[e] = (e % m == e / m) ? 1.0 : 0.0;
    if (c.V)
        for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += BNT) c.V[e] = (e % n == e / n) ? 1.0 : 0.0;
    __syncthreads();
    for (int64_t i = 0;; ++i) {
        const int64_t k0 = i * (int64_t)c.b;
        const int64_t np = c.n - k0;
        if (np <= 0) break;
        if (np <= c.b) {
            b_panel_and_svd<NT>(c, k0, (int)np, sm);
            break;
        }
        b_sketch_step<NT>(c, i, sm);
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_batched(BatchDesc* desc, const int* order, int count, int q, int prec,
                                                 double* slots, size_t slot_doubles, int64_t maxdim,
                                                 unsigned* next) {
    extern __shared__ double bsm_raw[];
    BSmem& sm = *reinterpret_cast<BSmem*>(bsm_raw);
    __shared__ int s_item;
    double* base = slots + (size_t)blockIdx.x * slot_doubles;
    const int64_t L = maxdim * BMAX;
    Slot s;
    s.G = base;
    s.Y = base + L;
    s.Z = base + 2 * L;
    s.W = base + 3 * L;
    s.X = base + 4 * L;
    s.X2 = base + 5 * L;
    s.tmp = base + 6 * L;
    s.tau = base + 7 * L;
    s.Tf = s.tau + BMAX;
    s.gram = s.Tf + BMAX * BMAX;
    s.D = s.gram + BMAX * BMAX;
    s.Us = s.D + BMAX;
    s.Vs = s.Us + BMAX * BMAX;
    s.Yf = (float*)(s.Vs + BMAX * BMAX);
    s.Zf = s.Yf + L;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned k = atomicAdd(next, 1u);
            s_item = (k < (unsigned)count) ? order[k] : -1;
        }
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item < 0) break;
        BatchDesc& d = desc[item];
        MatCtx c;
        c.m = d.m;
        c.n = d.n;
        c.b = d.b;
        c.q = q;
        c.prec = prec;
        c.tile = d.tile;
        c.seed = d.seed;
        c.U = d.U;
        c.T = d.T;
        c.V = d.V;
        c.s = s;
        c.status = &d.status;
        b_factor_one<NT>(c, d.A, d.lda, sm);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
double est_cost(int64_t m, int64_t n, int b, int q) {
    double F = 0.0;
    for (int64_t i = 0;; ++i) {
        int64_t mp = m - i * b, np = n - i * b;
        if (np <= 0) break;
        if (np <= b) {
            F += 2.0 * mp * np * np + 4.0 * m * mp * np;
            break;
        }
        F += 2.0 * (1 + 2 * q) * mp * np * b + 4.0 * m * np * b + 4.0 * mp * (np - b) * b + 4.0 * n * np * b +
             4.0 * m * mp * b;
    }
    return F;
}

__global__ void k_batched_reset(BatchDesc* desc, int count, unsigned* next) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) desc[i].status = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *next = 0u;
}

struct TuneRow {
    int64_t nmin, nmax;
    int tall, b, tile;
};

struct TuneTable {
    std::vector<TuneRow> rows;
    int threads = 256;  // threads per CTA, i.e. per matrix in flight
};

// Lines "nmin nmax tall b [tile]" (tile 32 or 64, default 64) and an
// optional line "threads NT" (128 or 256, default 256).
TuneTable parse_table(const char* text) {
    TuneTable t;
    if (!text) {  // built-in defaults (randutv_batched_autotune measures replacements)
        t.rows.push_back({0, 63, -1, 16, 32});
        t.rows.push_back({64, 191, -1, 32, 64});
        t.rows.push_back({192, 1LL << 40, -1, 64, 64});
        return t;
    }
    std::string all(text);
    size_t pos = 0;
    while (pos < all.size()) {
        size_t e = all.find('\n', pos);
        if (e == std::string::npos) e = all.size();
        const std::string line = all.substr(pos, e - pos);
        pos = e + 1;
        int nt = 0;
        if (sscanf(line.c_str(), " threads %d", &nt) == 1) {
            t.threads = (nt == 128) ? 128 : 256;
            continue;
        }
        long long a, bmax;
        int tall, b, tile = 64;
        const int got = sscanf(line.c_str(), "%lld %lld %d %d %d", &a, &bmax, &tall, &b, &tile);
        if (got >= 4) t.rows.push_back({a, bmax, tall, b, (got == 5 && tile == 32) ? 32 : 64});
    }
    return t;
}

// Block size and GEMM tile of an m x n matrix from the table.
void pick(const TuneTable& t, int64_t m, int64_t n, int* b, int* tile) {
    int tall = m > n ? 1 : 0;
    for (const TuneRow& r : t.rows)
        if (n >= r.nmin && n <= r.nmax && (r.tall < 0 || r.tall == tall)) {
            *b = std::min(std::max(r.b, 1), BMAX);
            *tile = r.tile;
            return;
        }
    *b = 32;
    *tile = 64;
}

}  // namespace

}  // namespace rutv

using namespace rutv;

// A prepared batch: descriptors and queue order resident on the device, one
// workspace slot per CTA, and a CUDA graph (status reset + persistent kernel)
// that every run replays.
struct randutv_batch_plan {
    int count = 0, q = 0, prec = 0, grid = 0, dev = 0, threads = 256;
    void* buf = nullptr;
    BatchDesc* ddesc = nullptr;
    int* host_status = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<BatchDesc> h;
};

namespace {

randutv_status plan_build(int count, const int64_t* m, const int64_t* n, const double* const* A, const int64_t* lda,
                          double* const* U, double* const* T, double* const* V, const uint64_t* seed, int q, int prec,
                          const int* bsel, const int* tsel, int threads, cudaStream_t st, randutv_batch_plan** out) {
    *out = nullptr;
    if (count <= 0 || q < 0) return RANDUTV_EINVAL;
    if (prec != RANDUTV_FP64 && prec != RANDUTV_SKETCH_FP32) return RANDUTV_ENOTIMPL;
    auto* P = new randutv_batch_plan();
    P->count = count;
    P->q = q;
    P->prec = prec;
    P->threads = (threads == 128) ? 128 : 256;
    int64_t maxdim = 1;
    P->h.resize(count);
    std::vector<std::pair<double, int>> cost(count);
    for (int i = 0; i < count; ++i) {
        if (m[i] < n[i] || n[i] < 0 || lda[i] < std::max<int64_t>(m[i], 1) || (n[i] > 0 && (!A[i] || !T[i])) ||
            m[i] > 8192) {
            delete P;
            return RANDUTV_EINVAL;
        }
        int b = std::min(std::max(bsel[i], 1), BMAX);
        P->h[i] = BatchDesc{m[i], n[i], lda[i], A[i], U ? U[i] : nullptr, T[i], V ? V[i] : nullptr,
                            seed ? seed[i] : 0, b, 0, (tsel && tsel[i] == 32) ? 32 : 64};
        maxdim = std::max(maxdim, m[i]);
        cost[i] = {est_cost(m[i], n[i], b, q), i};
    }
    std::sort(cost.begin(), cost.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first > b.first || (a.first == b.first && a.second < b.second);
    });
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = cost[i].second;

    if (cudaGetDevice(&P->dev) != cudaSuccess) { delete P; return RANDUTV_ECUDA; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->dev);
    const size_t shm = sizeof(BSmem);
    const void* kfn = (P->threads == 128) ? (const void*)k_batched<128> : (const void*)k_batched<256>;
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) {
        delete P;
        return RANDUTV_ECUDA;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, P->threads, shm);
    per_sm = std::max(1, std::min(per_sm, P->threads == 128 ? 4 : 2));
    P->grid = std::min(count, sms * per_sm);
    const int64_t L = maxdim * BMAX;
    const size_t slot_doubles = (size_t)7 * L + BMAX + 4 * (size_t)BMAX * BMAX + BMAX + (size_t)L + 64;
    const size_t slots_bytes = (sizeof(double) * slot_doubles * P->grid + 255) / 256 * 256;
    const size_t desc_bytes = (sizeof(BatchDesc) * count + 255) / 256 * 256;
    const size_t order_bytes = (sizeof(int) * count + 255) / 256 * 256;
    if (cudaMalloc(&P->buf, slots_bytes + desc_bytes + order_bytes + 256) != cudaSuccess) {
        delete P;
        return RANDUTV_ENOMEM;
    }
    char* p = (char*)P->buf;
    double* slots = (double*)p;
    P->ddesc = (BatchDesc*)(p + slots_bytes);
    int* dorder = (int*)(p + slots_bytes + desc_bytes);
    unsigned* next = (unsigned*)(p + slots_bytes + desc_bytes + order_bytes);
    if (cudaMemcpy(P->ddesc, P->h.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dorder, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
        randutv_batched_plan_destroy(P);
        return RANDUTV_ECUDA;
    }
    // capture: reset statuses and the queue head, then the persistent kernel
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        randutv_batched_plan_destroy(P);
        return RANDUTV_ECUDA;
    }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        k_batched_reset<<<std::max(1, std::min(64, (count + 255) / 256)), 256, 0, cs>>>(P->ddesc, count, next);
        if (P->threads == 128)
            k_batched<128><<<P->grid, 128, shm, cs>>>(P->ddesc, dorder, count, q, prec, slots, slot_doubles, maxdim,
                                                      next);
        else
            k_batched<256><<<P->grid, 256, shm, cs>>>(P->ddesc, dorder, count, q, prec, slots, slot_doubles, maxdim,
                                                      next);
        ok = cudaStreamEndCapture(cs, &P->graph) == cudaSuccess;
    }
    cudaStreamDestroy(cs);
    if (!ok || cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess) {
        randutv_batched_plan_destroy(P);
        return RANDUTV_ECUDA;
    }
    (void)st;
    *out = P;
    return RANDUTV_OK;
}

randutv_status plan_run(randutv_batch_plan* P, int* status, cudaStream_t st, float* ms_out) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    {
        TraceScope ts("batched", 0.0, 0.0, st);
        if (cudaGraphLaunch(P->exec, st) != cudaSuccess) return RANDUTV_ECUDA;
        trace_count(2);
    }
    if (ms_out) cudaEventRecord(e1, st);
    if (cudaMemcpyAsync(P->h.data(), P->ddesc, sizeof(BatchDesc) * P->count, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return RANDUTV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RANDUTV_ECUDA;
    if (ms_out) {
        cudaEventElapsedTime(ms_out, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int worst = 0;
    for (int i = 0; i < P->count; ++i) {
        int si = RANDUTV_OK;
        if (P->h[i].status & ST_NONFINITE) si = RANDUTV_ENONFINITE;
        else if (P->h[i].status & ST_NOCONV) si = RANDUTV_ENOCONV;
        if (status) status[i] = si;
        worst = std::max(worst, si);
    }
    return (randutv_status)worst;
}

}  // namespace

extern "C" {

randutv_status randutv_batched_plan_create(int count, const int64_t* m, const int64_t* n, const double* const* A,
                                           const int64_t* lda, double* const* U, double* const* T, double* const* V,
                                           const uint64_t* seed, int q, int prec, const char* autotune_table,
                                           randutv_batch_plan** plan) {
    if (!plan) return RANDUTV_EINVAL;
    *plan = nullptr;
    if (count <= 0 || !m || !n || !A || !lda || !T) return RANDUTV_EINVAL;
    const TuneTable tab = parse_table(autotune_table);
    std::vector<int> bsel(count), tsel(count);
    for (int i = 0; i < count; ++i) pick(tab, m[i], n[i], &bsel[i], &tsel[i]);
    return plan_build(count, m, n, A, lda, U, T, V, seed, q, prec, bsel.data(), tsel.data(), tab.threads, nullptr,
                      plan);
}

randutv_status randutv_batched_plan_run(randutv_batch_plan* plan, int* status, void* stream) {
    if (!plan) return RANDUTV_EINVAL;
    return plan_run(plan, status, (cudaStream_t)stream, nullptr);
}

void randutv_batched_plan_destroy(randutv_batch_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->buf) {
        cudaDeviceSynchronize();
        cudaFree(plan->buf);
    }
    delete plan;
}

randutv_status randutv_batched(int count, const int64_t* m, const int64_t* n, const double* const* A,
                               const int64_t* lda, double* const* U, double* const* T, double* const* V,
                               const uint64_t* seed, int q, int prec, const char* autotune_table, int* status,
                               void* stream) {
    if (count == 0) return RANDUTV_OK;
    randutv_batch_plan* P = nullptr;
    randutv_status r = randutv_batched_plan_create(count, m, n, A, lda, U, T, V, seed, q, prec, autotune_table, &P);
    if (r != RANDUTV_OK) return r;
    r = plan_run(P, status, (cudaStream_t)stream, nullptr);
    randutv_batched_plan_destroy(P);
    return r;
}

randutv_status randutv_batched_autotune(int count, const int64_t* m, const int64_t* n, const double* const* A,
                                        const int64_t* lda, double* const* U, double* const* T, double* const* V,
                                        const uint64_t* seed, int q, int prec, char* table_out, size_t table_bytes,
                                        void* stream) {
    if (count <= 0 || !m || !n || !A || !lda || !T || !table_out || table_bytes < 64) return RANDUTV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // times one plan over the members idx of the batch with per-member b and tile
    auto time_plan = [&](const std::vector<int>& idx, const std::vector<int>& bs, const std::vector<int>& ts,
                         int threads, float* ms) -> randutv_status {
        const size_t k = idx.size();
        std::vector<int64_t> sm_(k), sn(k), sl(k);
        std::vector<const double*> sA(k);
        std::vector<double*> sU(k), sT(k), sV(k);
        std::vector<uint64_t> ss(k);
        for (size_t t = 0; t < k; ++t) {
            const int i = idx[t];
            sm_[t] = m[i]; sn[t] = n[i]; sl[t] = lda[i]; sA[t] = A[i];
            sU[t] = U ? U[i] : nullptr; sT[t] = T[i]; sV[t] = V ? V[i] : nullptr; ss[t] = seed ? seed[i] : 0;
        }
        randutv_batch_plan* P = nullptr;
        randutv_status r = plan_build((int)k, sm_.data(), sn.data(), sA.data(), sl.data(), U ? sU.data() : nullptr,
                                      sT.data(), V ? sV.data() : nullptr, ss.data(), q, prec, bs.data(), ts.data(),
                                      threads, st, &P);
        if (r != RANDUTV_OK) return r;
        r = plan_run(P, nullptr, st, ms);
        randutv_batched_plan_destroy(P);
        return (r == RANDUTV_ENOCONV) ? RANDUTV_OK : r;
    };
    struct Choice {
        int64_t lo;
        int tall, b, tile;
    };
    std::vector<Choice> chosen;
    std::vector<int> bsel(count, 32), tsel(count, 64);
    const int bcands[3] = {16, 32, 64};
    const int tcands[2] = {32, 64};
    // per size class (n in [lo, 2 lo), square and tall apart): block size and GEMM tile
    for (int64_t lo = 1; lo <= (1LL << 20); lo <<= 1)
        for (int tall = 0; tall < 2; ++tall) {
            std::vector<int> idx;
            for (int i = 0; i < count; ++i)
                if (n[i] >= lo && n[i] <= 2 * lo - 1 && ((m[i] > n[i]) ? 1 : 0) == tall) idx.push_back(i);
            if (idx.empty()) continue;
            std::vector<int> all = idx;
            if (idx.size() > 608) idx.resize(608);  // a representative sample of the class
            Choice best{lo, tall, 32, 64};
            float best_ms = 1e30f;
            for (int b : bcands)
                for (int tile : tcands) {
                    float ms = 0.f;
                    randutv_status r = time_plan(idx, std::vector<int>(idx.size(), b),
                                                 std::vector<int>(idx.size(), tile), 256, &ms);
                    if (r != RANDUTV_OK) return r;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = Choice{lo, tall, b, tile};
                    }
                }
            chosen.push_back(best);
            for (int i : all) {
                bsel[i] = best.b;
                tsel[i] = best.tile;
            }
        }
    // threads per matrix: the whole batch with its chosen block sizes and tiles
    std::vector<int> every(count);
    for (int i = 0; i < count; ++i) every[i] = i;
    int best_threads = 256;
    float best_ms = 1e30f;
    for (int threads : {128, 256}) {
        float ms = 0.f;
        randutv_status r = time_plan(every, bsel, tsel, threads, &ms);
        if (r != RANDUTV_OK) return r;
        if (ms < best_ms) {
            best_ms = ms;
            best_threads = threads;
        }
    }
    std::string out;
    for (const Choice& ch : chosen) {
        char line[96];
        snprintf(line, sizeof(line), "%lld %lld %d %d %d\n", (long long)ch.lo, (long long)(2 * ch.lo - 1), ch.tall,
                 ch.b, ch.tile);
        out += line;
    }
    out += "threads " + std::to_string(best_threads) + "\n";
    if (out.size() + 1 > table_bytes) return RANDUTV_ENOMEM;
    memcpy(table_out, out.c_str(), out.size() + 1);
    return RANDUTV_OK;
}

}  // extern "C"
