/*
 * randutv_oracle.c -- plain, slow, FP64 CPU oracle for the blocked randUTV
 * factorization A = U T V^T (Heavner, Igual, Quintana-Orti, Martinsson,
 * "Efficient algorithms for computing a rank-revealing UTV factorization on
 * parallel computing architectures", arXiv 2104.05782).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker of the CUDA path: only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library
 * and never calls it.
 *
 * Every routine is the textbook definition written out with plain loops,
 * column-major storage, FP64 arithmetic.  The only parallelism is an OpenMP
 * loop over independent output columns, which does not change the order in
 * which any single output entry is summed.
 *
 * Where the paper is silent these readings are taken (all restated in the
 * design notes of the repository):
 *   - the Gaussian matrix G of Sec. 3.2.1 is drawn from a counter-based
 *     generator, Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), followed by
 *     the Box-Muller transform (see oracle_gaussian);
 *   - Householder vectors follow LAPACK's dlarfg sign convention (Sec. 2.2
 *     only says "HQR");
 *   - the b x b SVD of Sec. 3.2.3 is a one-sided (Hestenes) Jacobi SVD, with
 *     singular values sorted descending and each singular pair signed so that
 *     the entry of largest modulus of the right vector is positive;
 *   - the right update with V_alpha covers all m rows of T(:, J2) (Sec. 5.4 and
 *     the Matlab listing of Sec. 3.2), the left update is (I - W T W^T)^T C;
 *   - when at most b columns remain the trailing block is factorised without a
 *     sketch (panel QR + small SVD), as the Matlab listing of Sec. 3.2 does with
 *     a full SVD.
 *
 * Parity pins (tests/test_oracle_*.py): Philox against numpy's Philox bit
 * generator; Householder QR against LAPACK dgeqrf; the T factor against LAPACK
 * dgeqrt and against the explicit product of reflectors; Jacobi SVD against
 * LAPACK singular values; the whole factorization against the identities that
 * define a UTV factorization and against brute-force SVD on tiny inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------- */
/* Philox4x64-10, from its published definition (Salmon et al., SC'11):     */
/* ten rounds of two 64x64->128 multiplies, the key bumped by the Weyl       */
/* constants between rounds.                                                 */
/* ------------------------------------------------------------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* G^(i)(r, c) of Sec. 3.2.1 (i.i.d. N(0,1)).  Counter = (r / 4, c, i, 0),
 * key = (seed, 0).  Each 64-bit word x gives u = (floor(x / 2^11) + 1) * 2^-53
 * in (0, 1]; words (0,1) and (2,3) are Box-Muller pairs:
 *   z_even = sqrt(-2 ln u_a) cos(2 pi u_b),  z_odd = sqrt(-2 ln u_a) sin(2 pi u_b),
 * giving rows 4k, 4k+1 (first pair) and 4k+2, 4k+3 (second pair). */
void oracle_gaussian(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G, int64_t ldg) {
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    for (int64_t c = 0; c < cols; ++c) {
        for (int64_t k = 0; 4 * k < rows; ++k) {
            uint64_t ctr[4] = {(uint64_t)k, (uint64_t)c, (uint64_t)step, 0};
            uint64_t key[2] = {seed, 0};
            uint64_t x[4];
            oracle_philox4x64_10(ctr, key, x);
            double u[4];
            for (int t = 0; t < 4; ++t) u[t] = ((double)(x[t] >> 11) + 1.0) * inv53;
            double z[4];
            for (int pair = 0; pair < 2; ++pair) {
                double rad = sqrt(-2.0 * log(u[2 * pair]));
                double ang = two_pi * u[2 * pair + 1];
                z[2 * pair] = rad * cos(ang);
                z[2 * pair + 1] = rad * sin(ang);
            }
            for (int t = 0; t < 4; ++t) {
                int64_t r = 4 * k + t;
                if (r < rows) G[IDX(r, c, ldg)] = z[t];
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Plain matrix product C := alpha * op(A) op(B) + beta * C (definition).    */
/* ------------------------------------------------------------------------- */
void oracle_gemm(int transA, int transB, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        for (int64_t i = 0; i < M; ++i) {
            double s = 0.0;
            for (int64_t l = 0; l < K; ++l) {
                double a = transA ? A[IDX(l, i, lda)] : A[IDX(i, l, lda)];
                double b = transB ? B[IDX(j, l, ldb)] : B[IDX(l, j, ldb)];
                s += a * b;
            }
            C[IDX(i, j, ldc)] = (beta == 0.0 ? 0.0 : beta * C[IDX(i, j, ldc)]) + alpha * s;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Unpivoted Householder QR (HQR, Sec. 2.2), one reflector per column, each  */
/* built with LAPACK's dlarfg rule:                                          */
/*   alpha = A(j,j), x = A(j+1:M, j), xi = ||x||_2;                          */
/*   xi == 0  -> tau = 0 (H = I), A(j,j) unchanged;                          */
/*   else beta = -sign(alpha) hypot(alpha, xi) (sign(+-0) = +),              */
/*        tau = (beta - alpha) / beta, v = [1; x / (alpha - beta)],          */
/*        A(j,j) = beta.                                                     */
/* H_j = I - tau v v^T is applied to A(j:M, j+1:N).  On exit R is on and     */
/* above the diagonal, the unit lower Householder vectors W below it.        */
/* ------------------------------------------------------------------------- */
void oracle_householder_qr(int64_t M, int64_t N, double* A, int64_t lda, double* tau) {
    int64_t kmax = M < N ? M : N;
    for (int64_t j = 0; j < kmax; ++j) {
        double alpha = A[IDX(j, j, lda)];
        double xi2 = 0.0;
        for (int64_t r = j + 1; r < M; ++r) xi2 += A[IDX(r, j, lda)] * A[IDX(r, j, lda)];
        double xi = sqrt(xi2);
        if (xi == 0.0) {
            tau[j] = 0.0;
            continue;
        }
        double h = hypot(alpha, xi);
        double beta = (alpha >= 0.0) ? -h : h;
        tau[j] = (beta - alpha) / beta;
        double denom = alpha - beta;
        for (int64_t r = j + 1; r < M; ++r) A[IDX(r, j, lda)] /= denom;
        A[IDX(j, j, lda)] = beta;
        /* apply H_j to the columns right of j: A := A - tau v (v^T A) */
#pragma omp parallel for schedule(static)
        for (int64_t c = j + 1; c < N; ++c) {
            double w = A[IDX(j, c, lda)];
            for (int64_t r = j + 1; r < M; ++r) w += A[IDX(r, j, lda)] * A[IDX(r, c, lda)];
            w *= tau[j];
            A[IDX(j, c, lda)] -= w;
            for (int64_t r = j + 1; r < M; ++r) A[IDX(r, c, lda)] -= w * A[IDX(r, j, lda)];
        }
    }
}

/* Copy the unit lower trapezoidal Householder vectors (M x k) out of the QR
 * storage into a dense W. */
static void extract_w(int64_t M, int64_t k, const double* A, int64_t lda, double* W, int64_t ldw) {
    for (int64_t j = 0; j < k; ++j)
        for (int64_t r = 0; r < M; ++r)
            W[IDX(r, j, ldw)] = (r < j) ? 0.0 : (r == j ? 1.0 : A[IDX(r, j, lda)]);
}

/* ------------------------------------------------------------------------- */
/* Triangular factor of the compact WY form (Sec. 2.3): with                  */
/* Q = H_0 H_1 ... H_{k-1}, H_j = I - tau_j w_j w_j^T, find upper triangular  */
/* Tf with Q = I - W Tf W^T.  Forward, column by column:                     */
/*   Tf(j,j) = tau_j,  Tf(0:j, j) = -tau_j Tf(0:j,0:j) (W(:,0:j)^T w_j).      */
/* W is dense unit lower trapezoidal (M x k).                                */
/* ------------------------------------------------------------------------- */
void oracle_larft(int64_t M, int64_t k, const double* W, int64_t ldw, const double* tau, double* Tf,
                  int64_t ldt) {
    double* z = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t j = 0; j < k; ++j) {
        for (int64_t i = 0; i < k; ++i) Tf[IDX(i, j, ldt)] = 0.0;
        for (int64_t i = 0; i < j; ++i) {
            double s = 0.0;
            for (int64_t r = 0; r < M; ++r) s += W[IDX(r, i, ldw)] * W[IDX(r, j, ldw)];
            z[i] = -tau[j] * s;
        }
        for (int64_t i = 0; i < j; ++i) {
            double s = 0.0;
            for (int64_t l = i; l < j; ++l) s += Tf[IDX(i, l, ldt)] * z[l];
            Tf[IDX(i, j, ldt)] = s;
        }
        Tf[IDX(j, j, ldt)] = tau[j];
    }
    free(z);
}

/* C (R x M) := C (I - W Tf W^T): the three products of Sec. 2.3. */
static void apply_wy_right(int64_t R, int64_t M, int64_t k, double* C, int64_t ldc, const double* W,
                           int64_t ldw, const double* Tf, int64_t ldt) {
    if (R == 0 || M == 0 || k == 0) return;
    double* X = (double*)malloc(sizeof(double) * (size_t)R * (size_t)k);
    double* X2 = (double*)malloc(sizeof(double) * (size_t)R * (size_t)k);
    oracle_gemm(0, 0, R, k, M, 1.0, C, ldc, W, ldw, 0.0, X, R);      /* X = C W      */
    oracle_gemm(0, 0, R, k, k, 1.0, X, R, Tf, ldt, 0.0, X2, R);      /* X2 = X Tf    */
    oracle_gemm(0, 1, R, M, k, -1.0, X2, R, W, ldw, 1.0, C, ldc);    /* C -= X2 W^T  */
    free(X);
    free(X2);
}

/* C (M x N) := (I - W Tf W^T)^T C = C - W Tf^T (W^T C). */
static void apply_wy_left_t(int64_t M, int64_t N, int64_t k, double* C, int64_t ldc, const double* W,
                            int64_t ldw, const double* Tf, int64_t ldt) {
    if (M == 0 || N == 0 || k == 0) return;
    double* X = (double*)malloc(sizeof(double) * (size_t)k * (size_t)N);
    double* X2 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)N);
    oracle_gemm(1, 0, k, N, M, 1.0, W, ldw, C, ldc, 0.0, X, k);      /* X = W^T C    */
    oracle_gemm(1, 0, k, N, k, 1.0, Tf, ldt, X, k, 0.0, X2, k);      /* X2 = Tf^T X  */
    oracle_gemm(0, 0, M, N, k, -1.0, W, ldw, X2, k, 1.0, C, ldc);    /* C -= W X2    */
    free(X);
    free(X2);
}

/* ------------------------------------------------------------------------- */
/* One-sided (Hestenes) Jacobi SVD of an n x n matrix R = Us diag(D) Vs^T.    */
/* Cyclic-by-rows sweeps over column pairs (p, q); a pair is rotated when    */
/* |a_p^T a_q| > tol sqrt(|a_p|^2 |a_q|^2), tol = n 2^-53; the rotation is   */
/* the one that makes the two columns orthogonal (Golub & Van Loan, Sec.      */
/* 8.6): zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| +        */
/* sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t.  Converged when a sweep     */
/* rotates nothing; at most max_sweeps sweeps (else returns 1).              */
/* Then D(j) = |a_j|, Us(:,j) = a_j / D(j) (columns with D = 0 are completed */
/* by Gram-Schmidt on the unit vectors), sorted by D descending (stable),    */
/* and each pair (Us(:,j), Vs(:,j)) negated when the entry of largest        */
/* modulus of Vs(:,j) (lowest index on ties) is negative.                    */
/* ------------------------------------------------------------------------- */
int oracle_jacobi_svd(int64_t n, const double* R, int64_t ldr, double* D, double* Us, int64_t ldu,
                      double* Vs, int64_t ldv, int max_sweeps, int* sweeps_out) {
    if (n <= 0) { if (sweeps_out) *sweeps_out = 0; return 0; }
    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            A[IDX(i, j, n)] = R[IDX(i, j, ldr)];
            V[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
        }
    const double tol = (double)n * 1.1102230246251565e-16;
    int sweep = 0, converged = 0;
    while (sweep < max_sweeps) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p)
            for (int64_t q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t r = 0; r < n; ++r) {
                    double ap = A[IDX(r, p, n)], aq = A[IDX(r, q, n)];
                    alpha += ap * ap;
                    beta += aq * aq;
                    gamma += ap * aq;
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int64_t r = 0; r < n; ++r) {
                    double ap = A[IDX(r, p, n)], aq = A[IDX(r, q, n)];
                    A[IDX(r, p, n)] = c * ap - s * aq;
                    A[IDX(r, q, n)] = s * ap + c * aq;
                    double vp = V[IDX(r, p, n)], vq = V[IDX(r, q, n)];
                    V[IDX(r, p, n)] = c * vp - s * vq;
                    V[IDX(r, q, n)] = s * vp + c * vq;
                }
            }
        ++sweep;
        if (!rotated) { converged = 1; break; }
    }
    if (sweeps_out) *sweeps_out = sweep;
    /* singular values = column norms; order descending, stable */
    double* norms = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t r = 0; r < n; ++r) s += A[IDX(r, j, n)] * A[IDX(r, j, n)];
        norms[j] = sqrt(s);
        order[j] = j;
    }
    for (int64_t a = 1; a < n; ++a) { /* insertion sort: stable */
        int64_t key = order[a];
        int64_t b = a - 1;
        while (b >= 0 && norms[order[b]] < norms[key]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = key;
    }
    for (int64_t j = 0; j < n; ++j) {
        int64_t src = order[j];
        D[j] = norms[src];
        for (int64_t r = 0; r < n; ++r) {
            Vs[IDX(r, j, ldv)] = V[IDX(r, src, n)];
            Us[IDX(r, j, ldu)] = (norms[src] > 0.0) ? A[IDX(r, src, n)] / norms[src] : 0.0;
        }
    }
    /* complete the left vectors of zero singular values (Gram-Schmidt, twice) */
    for (int64_t j = 0; j < n; ++j) {
        if (D[j] > 0.0) continue;
        for (int64_t e = 0; e < n; ++e) {
            for (int64_t r = 0; r < n; ++r) Us[IDX(r, j, ldu)] = (r == e) ? 1.0 : 0.0;
            for (int pass = 0; pass < 2; ++pass)
                for (int64_t l = 0; l < n; ++l) {
                    if (l == j || (D[l] == 0.0 && l > j)) continue;
                    double d = 0.0;
                    for (int64_t r = 0; r < n; ++r) d += Us[IDX(r, l, ldu)] * Us[IDX(r, j, ldu)];
                    for (int64_t r = 0; r < n; ++r) Us[IDX(r, j, ldu)] -= d * Us[IDX(r, l, ldu)];
                }
            double nn = 0.0;
            for (int64_t r = 0; r < n; ++r) nn += Us[IDX(r, j, ldu)] * Us[IDX(r, j, ldu)];
            nn = sqrt(nn);
            if (nn > 0.5) {
                for (int64_t r = 0; r < n; ++r) Us[IDX(r, j, ldu)] /= nn;
                break;
            }
        }
    }
    /* canonical sign */
    for (int64_t j = 0; j < n; ++j) {
        int64_t imax = 0;
        double vmax = -1.0;
        for (int64_t r = 0; r < n; ++r)
            if (fabs(Vs[IDX(r, j, ldv)]) > vmax) { vmax = fabs(Vs[IDX(r, j, ldv)]); imax = r; }
        if (Vs[IDX(imax, j, ldv)] < 0.0)
            for (int64_t r = 0; r < n; ++r) {
                Vs[IDX(r, j, ldv)] = -Vs[IDX(r, j, ldv)];
                Us[IDX(r, j, ldu)] = -Us[IDX(r, j, ldu)];
            }
    }
    free(norms);
    free(order);
    free(A);
    free(V);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------------- */
/* Panel step shared by the sketch step and the final block (Sec. 3.2.2 and  */
/* Sec. 3.2.3): at column offset k0, factor the m' x w panel T(k0:m, k0:k0+w) */
/* by HQR; apply (I - W Tf W^T)^T to T(k0:m, k0+w:n) and (I - W Tf W^T) from  */
/* the right to U(:, k0:m); then the w x w SVD of R = Us D Vs^T:              */
/* T(k0:k0+w, k0:k0+w) = diag(D), T(0:k0, blk) *= Vs, T(blk, k0+w:n) =        */
/* Us^T T(blk, k0+w:n), V(:, blk) *= Vs, U(:, blk) *= Us; zero T below the    */
/* diagonal block.                                                            */
/* ------------------------------------------------------------------------- */
static int panel_and_svd(int64_t m, int64_t n, int64_t k0, int64_t w, double* T, double* U, double* V,
                         int max_sweeps) {
    int64_t mp = m - k0;
    double* tau = (double*)calloc((size_t)w, sizeof(double));
    double* W = (double*)malloc(sizeof(double) * (size_t)mp * (size_t)w);
    double* Tf = (double*)malloc(sizeof(double) * (size_t)w * (size_t)w);
    double* Pnl = T + IDX(k0, k0, m);
    oracle_householder_qr(mp, w, Pnl, m, tau);
    extract_w(mp, w, Pnl, m, W, mp);
    oracle_larft(mp, w, W, mp, tau, Tf, w);
    /* T22(:, w:) := (I - W Tf W^T)^T T22(:, w:) */
    apply_wy_left_t(mp, n - k0 - w, w, T + IDX(k0, k0 + w, m), m, W, mp, Tf, w);
    /* U(:, k0:m) := U(:, k0:m) (I - W Tf W^T) */
    if (U) apply_wy_right(m, mp, w, U + IDX(0, k0, m), m, W, mp, Tf, w);
    /* small SVD of the upper triangular R */
    double* R = (double*)malloc(sizeof(double) * (size_t)w * (size_t)w);
    for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < w; ++i) R[IDX(i, j, w)] = (i <= j) ? Pnl[IDX(i, j, m)] : 0.0;
    double* D = (double*)malloc(sizeof(double) * (size_t)w);
    double* Us = (double*)malloc(sizeof(double) * (size_t)w * (size_t)w);
    double* Vs = (double*)malloc(sizeof(double) * (size_t)w * (size_t)w);
    int rc = oracle_jacobi_svd(w, R, w, D, Us, w, Vs, w, max_sweeps, NULL);
    /* T(0:k0, blk) := T(0:k0, blk) Vs */
    if (k0 > 0) {
        double* X = (double*)malloc(sizeof(double) * (size_t)k0 * (size_t)w);
        oracle_gemm(0, 0, k0, w, w, 1.0, T + IDX(0, k0, m), m, Vs, w, 0.0, X, k0);
        for (int64_t j = 0; j < w; ++j)
            for (int64_t i = 0; i < k0; ++i) T[IDX(i, k0 + j, m)] = X[IDX(i, j, k0)];
        free(X);
    }
    /* T(blk, k0+w:n) := Us^T T(blk, k0+w:n) */
    int64_t nr = n - k0 - w;
    if (nr > 0) {
        double* X = (double*)malloc(sizeof(double) * (size_t)w * (size_t)nr);
        oracle_gemm(1, 0, w, nr, w, 1.0, Us, w, T + IDX(k0, k0 + w, m), m, 0.0, X, w);
        for (int64_t j = 0; j < nr; ++j)
            for (int64_t i = 0; i < w; ++i) T[IDX(k0 + i, k0 + w + j, m)] = X[IDX(i, j, w)];
        free(X);
    }
    /* diagonal block := diag(D); zero the panel below it */
    for (int64_t j = 0; j < w; ++j)
        for (int64_t i = k0; i < m; ++i) T[IDX(i, k0 + j, m)] = (i == k0 + j) ? D[j] : 0.0;
    if (V) {
        double* X = (double*)malloc(sizeof(double) * (size_t)n * (size_t)w);
        oracle_gemm(0, 0, n, w, w, 1.0, V + IDX(0, k0, n), n, Vs, w, 0.0, X, n);
        for (int64_t j = 0; j < w; ++j)
            for (int64_t i = 0; i < n; ++i) V[IDX(i, k0 + j, n)] = X[IDX(i, j, n)];
        free(X);
    }
    if (U) {
        double* X = (double*)malloc(sizeof(double) * (size_t)m * (size_t)w);
        oracle_gemm(0, 0, m, w, w, 1.0, U + IDX(0, k0, m), m, Us, w, 0.0, X, m);
        for (int64_t j = 0; j < w; ++j)
            for (int64_t i = 0; i < m; ++i) U[IDX(i, k0 + j, m)] = X[IDX(i, j, m)];
        free(X);
    }
    free(tau); free(W); free(Tf); free(R); free(D); free(Us); free(Vs);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* randUTV (Sec. 3.2 outline; Sec. 3.2.1-3.2.3; Householder/compact-WY form   */
/* of the FLAME algorithm of Sec. 4.3).                                      */
/*   T := A, U := I_m, V := I_n.                                             */
/*   For i = 0, 1, ...: k0 = i b, m' = m - k0, n' = n - k0.                  */
/*     n' > b:  G (m' x b) Gaussian; Y := T22^T G; q times Y := T22^T(T22 Y) */
/*              HQR(Y) -> W_V, Tf_V; T(:, k0:n) := T(:, k0:n)(I - W Tf W^T)  */
/*              (all m rows); V(:, k0:n) likewise; then panel_and_svd(b).    */
/*     0 < n' <= b: panel_and_svd(n') and stop.                              */
/* U and/or V may be NULL ("no orthonormal matrices" mode).  stop_after >= 0 */
/* stops after that many block steps (the partial factorization is still an  */
/* exact UTV of A).  m >= n >= 0, b >= 1, q >= 0 are required.               */
/* Returns 0, or 1 when a Jacobi SVD hit its sweep cap, or -1 on bad input.  */
/* ------------------------------------------------------------------------- */
int oracle_randutv(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int64_t q, uint64_t seed,
                   double* U, double* T, double* V, int64_t stop_after, int max_sweeps) {
    if (m < n || n < 0 || b < 1 || q < 0 || lda < m) return -1;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) T[IDX(i, j, m)] = A[IDX(i, j, lda)];
    if (U)
        for (int64_t j = 0; j < m; ++j)
            for (int64_t i = 0; i < m; ++i) U[IDX(i, j, m)] = (i == j) ? 1.0 : 0.0;
    if (V)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) V[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
    int status = 0;
    for (int64_t i = 0;; ++i) {
        if (stop_after >= 0 && i >= stop_after) break;
        int64_t k0 = i * b;
        int64_t np = n - k0, mp = m - k0;
        if (np <= 0) break;
        if (np <= b) {
            if (panel_and_svd(m, n, k0, np, T, U, V, max_sweeps)) status = 1;
            break;
        }
        double* T22 = T + IDX(k0, k0, m);
        double* G = (double*)malloc(sizeof(double) * (size_t)mp * (size_t)b);
        double* Y = (double*)malloc(sizeof(double) * (size_t)np * (size_t)b);
        double* Z = (double*)malloc(sizeof(double) * (size_t)mp * (size_t)b);
        oracle_gaussian(seed, i, mp, b, G, mp);
        oracle_gemm(1, 0, np, b, mp, 1.0, T22, m, G, mp, 0.0, Y, np);       /* Y = T22^T G */
        for (int64_t it = 0; it < q; ++it) {
            oracle_gemm(0, 0, mp, b, np, 1.0, T22, m, Y, np, 0.0, Z, mp);   /* Z = T22 Y   */
            oracle_gemm(1, 0, np, b, mp, 1.0, T22, m, Z, mp, 0.0, Y, np);   /* Y = T22^T Z */
        }
        double* tau = (double*)calloc((size_t)b, sizeof(double));
        double* W = (double*)malloc(sizeof(double) * (size_t)np * (size_t)b);
        double* Tf = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
        oracle_householder_qr(np, b, Y, np, tau);
        extract_w(np, b, Y, np, W, np);
        oracle_larft(np, b, W, np, tau, Tf, b);
        apply_wy_right(m, np, b, T + IDX(0, k0, m), m, W, np, Tf, b);
        if (V) apply_wy_right(n, np, b, V + IDX(0, k0, n), n, W, np, Tf, b);
        free(G); free(Y); free(Z); free(tau); free(W); free(Tf);
        if (panel_and_svd(m, n, k0, b, T, U, V, max_sweeps)) status = 1;
    }
    return status;
}

/* ------------------------------------------------------------------------- */
/* randUTV with a QR first, for tall inputs (Sec. 5.1: when m is much larger  */
/* than n the input is first reduced by an unpivoted QR and randUTV runs on   */
/* the n x n triangular factor).                                              */
/*   A = Q_A [R; 0]   (HQR of A, Sec. 2.2, the dlarfg rule as above),         */
/*   R = U_R T_R V^T  (oracle_randutv on the n x n R, same b, q, seed),      */
/*   T = [T_R; 0],  V = V,  U = Q_A diag(U_R, I_{m-n}).                       */
/* U is formed from its definition: X := diag(U_R, I), then the reflectors    */
/* H_j = I - tau_j v_j v_j^T (v_j = [0; 1; A(j+1:m, j)] of the QR storage)    */
/* are applied from the left, X := H_j X, for j = n-1 down to 0, since        */
/* Q_A = H_0 H_1 ... H_{n-1}.  U and/or V may be NULL; stop_after and         */
/* max_sweeps are passed to the randUTV of R.  Same return values as          */
/* oracle_randutv.                                                            */
/* ------------------------------------------------------------------------- */
int oracle_randutv_qrfirst(int64_t m, int64_t n, const double* A, int64_t lda, int64_t b, int64_t q,
                           uint64_t seed, double* U, double* T, double* V, int64_t stop_after, int max_sweeps) {
    if (m < n || n < 0 || b < 1 || q < 0 || lda < m) return -1;
    double* F = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
    double* tau = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* R = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
    double* TR = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
    double* UR = U ? (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1)) : NULL;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) F[IDX(i, j, m)] = A[IDX(i, j, lda)];
    oracle_householder_qr(m, n, F, m, tau);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) R[IDX(i, j, n)] = (i <= j) ? F[IDX(i, j, m)] : 0.0;
    int status = oracle_randutv(n, n, R, n, b, q, seed, UR, TR, V, stop_after, max_sweeps);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) T[IDX(i, j, m)] = (i < n) ? TR[IDX(i, j, n)] : 0.0;
    if (U) {
        for (int64_t j = 0; j < m; ++j)
            for (int64_t i = 0; i < m; ++i)
                U[IDX(i, j, m)] = (i < n && j < n) ? UR[IDX(i, j, n)] : (i == j && i >= n ? 1.0 : 0.0);
        for (int64_t j = n - 1; j >= 0; --j) {
            if (tau[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < m; ++c) {
                double s = U[IDX(j, c, m)];
                for (int64_t r = j + 1; r < m; ++r) s += F[IDX(r, j, m)] * U[IDX(r, c, m)];
                s *= tau[j];
                U[IDX(j, c, m)] -= s;
                for (int64_t r = j + 1; r < m; ++r) U[IDX(r, c, m)] -= s * F[IDX(r, j, m)];
            }
        }
    }
    free(F); free(tau); free(R); free(TR); free(UR);
    return status;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
