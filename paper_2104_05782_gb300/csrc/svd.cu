// svd.cu -- SVD of the b x b diagonal block by one-sided (Hestenes) Jacobi.
//
// Sec. 3.2.3 diagonalises T22(1:b, 1:b) = U_svd D V_svd^T to build V_beta and
// U_beta; the paper names no SVD method.  One-sided Jacobi is used because it
// keeps relative accuracy for tiny singular values and has a fixed, parallel
// pair schedule.  A pair of columns (p, q) is rotated when
// |a_p^T a_q| > tol sqrt(|a_p|^2 |a_q|^2), tol = w 2^-53, by the rotation that
// makes them orthogonal (zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t).
// Sweeps stop when no pair is rotated (cap: max_sweeps, else ST_NOCONV).
// Output is canonical: singular values descending (stable on ties), columns of
// Us = a_j / |a_j| (Gram-Schmidt completion for zero values), and each pair
// negated when the entry of largest modulus of Vs(:, j) (lowest index on
// ties) is negative.
//
// GB300 design: FP64 runs at ~7 GFLOP/s per SM, so a single block would need
// tens of milliseconds for b = 128.  The w/2 disjoint pairs of every round of
// a round-robin ("circle") ordering are instead spread over w/2 blocks of one
// cooperative launch, one pair per block, one row per thread, with A and V
// resident in L2; one grid barrier separates rounds.  The pair order differs
// from a cyclic-by-rows sweep, which changes only rounding: the converged,
// canonical SVD is the same.
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

__device__ __forceinline__ int circle_elem(int pos, int round, int n2) {
    return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n2 - 1);
}

template <int NT>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* red) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[warp * 3 + 0] = a;
        red[warp * 3 + 1] = b;
        red[warp * 3 + 2] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
    for (int k = 0; k < NT / 32; ++k) {
        a += red[k * 3 + 0];
        b += red[k * 3 + 1];
        c += red[k * 3 + 2];
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_jacobi(const double* __restrict__ R, int64_t ldr, int w, int n2,
                                               double* __restrict__ A, double* __restrict__ V,
                                               double* __restrict__ D, double* __restrict__ Us,
                                               double* __restrict__ Vs, unsigned* bar, int* rot, int* status,
                                               int max_sweeps, double tol) {
    __shared__ double red[3 * (NT / 32)];
    __shared__ int s_flag;
    const int tid = threadIdx.x, G = gridDim.x, cta = blockIdx.x;
    unsigned target = 0;

    // A := upper triangle of R, V := I (ld w)
    for (int c = cta; c < w; c += G)
        for (int r = tid; r < w; r += NT) {
            A[r + (size_t)c * w] = (r <= c) ? R[r + (int64_t)c * ldr] : 0.0;
            V[r + (size_t)c * w] = (r == c) ? 1.0 : 0.0;
        }
    if (cta == 0 && tid < 3) rot[tid] = 0;
    if (!grid_sync(bar, target, status)) return;

    bool converged = (w <= 1);
    int sweep = 0;
    for (; sweep < max_sweeps && !converged; ++sweep) {
        if (cta == 0 && tid == 0) rot[(sweep + 1) % 3] = 0;
        for (int round = 0; round < n2 - 1; ++round) {
            int p = circle_elem(cta, round, n2);
            int q = circle_elem(n2 - 1 - cta, round, n2);
            if (p > q) { int t = p; p = q; q = t; }
            if (q < w) {  // a pair with the padding column (odd w) is skipped
                double* ap = A + (size_t)p * w;
                double* aq = A + (size_t)q * w;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = tid; r < w; r += NT) {
                    double x = __ldcg(ap + r), y = __ldcg(aq + r);
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                block_sum3<NT>(al, be, ga, red);
                if (!isfinite(al) || !isfinite(be) || !isfinite(ga)) {
                    if (tid == 0) atomicOr(status, ST_NONFINITE);
                } else if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
                    double zeta = (be - al) / (2.0 * ga);
                    double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double cs = 1.0 / sqrt(1.0 + t * t);
                    double sn = cs * t;
                    double* vp = V + (size_t)p * w;
                    double* vq = V + (size_t)q * w;
                    for (int r = tid; r < w; r += NT) {
                        double x = __ldcg(ap + r), y = __ldcg(aq + r);
                        ap[r] = cs * x - sn * y;
                        aq[r] = sn * x + cs * y;
                        double u = __ldcg(vp + r), z = __ldcg(vq + r);
                        vp[r] = cs * u - sn * z;
                        vq[r] = sn * u + cs * z;
                    }
                    if (tid == 0) atomicAdd(rot + (sweep % 3), 1);
                }
            }
            if (!grid_sync(bar, target, status)) return;
        }
        if (tid == 0) s_flag = __ldcg(rot + (sweep % 3));
        __syncthreads();
        converged = (s_flag == 0);
    }
    if (cta != 0) return;
    if (!converged && tid == 0) atomicOr(status, ST_NOCONV);

    // ---- canonical output (block 0) ----------------------------------------
    // D[rank(c)] = |a_c|, rank = stable descending order
    extern __shared__ double nrm[];  // w doubles
    for (int c = tid; c < w; c += NT) {
        double s = 0.0;
        for (int r = 0; r < w; ++r) {
            double x = __ldcg(A + r + (size_t)c * w);
            s += x * x;
        }
        nrm[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < w; c += NT) {
        double v = nrm[c];
        int rank = 0;
        for (int c2 = 0; c2 < w; ++c2) {
            double u = nrm[c2];
            rank += (u > v) || (u == v && c2 < c);
        }
        D[rank] = v;
        for (int r = 0; r < w; ++r) {
            Vs[r + (size_t)rank * w] = __ldcg(V + r + (size_t)c * w);
            Us[r + (size_t)rank * w] = (v > 0.0) ? __ldcg(A + r + (size_t)c * w) / v : 0.0;
        }
    }
    __syncthreads();
    // left vectors of zero singular values: Gram-Schmidt (twice) on unit vectors
    if (tid == 0) {
        for (int j = 0; j < w; ++j) {
            if (D[j] > 0.0) continue;
            for (int e = 0; e < w; ++e) {
                double* u = Us + (size_t)j * w;
                for (int r = 0; r < w; ++r) u[r] = (r == e) ? 1.0 : 0.0;
                for (int pass = 0; pass < 2; ++pass)
                    for (int l = 0; l < w; ++l) {
                        if (l == j || (D[l] == 0.0 && l > j)) continue;
                        const double* ul = Us + (size_t)l * w;
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
    for (int j = tid; j < w; j += NT) {
        int imax = 0;
        double vmax = -1.0;
        for (int r = 0; r < w; ++r) {
            double a = fabs(Vs[r + (size_t)j * w]);
            if (a > vmax) { vmax = a; imax = r; }
        }
        if (Vs[imax + (size_t)j * w] < 0.0)
            for (int r = 0; r < w; ++r) {
                Vs[r + (size_t)j * w] = -Vs[r + (size_t)j * w];
                Us[r + (size_t)j * w] = -Us[r + (size_t)j * w];
            }
    }
}

}  // namespace

size_t jacobi_scratch_elems(int w) { return (size_t)2 * w * w; }

cudaError_t jacobi_svd(const double* R, int64_t ldr, int w, double* D, double* Us, double* Vs, double* scratch,
                       unsigned* bar, int* counters, int* status, int max_sweeps, cudaStream_t st) {
    if (w <= 0) return cudaSuccess;
    int n2 = w + (w & 1);
    int G = std::max(1, n2 / 2);
    double* A = scratch;
    double* V = scratch + (size_t)w * w;
    double tol = (double)w * 1.1102230246251565e-16;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    size_t shm = sizeof(double) * (size_t)w;
    void* args[] = {(void*)&R, (void*)&ldr, (void*)&w, (void*)&n2, (void*)&A, (void*)&V, (void*)&D,
                    (void*)&Us, (void*)&Vs, (void*)&bar, (void*)&counters, (void*)&status,
                    (void*)&max_sweeps, (void*)&tol};
    trace_count(1);
    if (w <= 128)
        return cudaLaunchCooperativeKernel((const void*)k_jacobi<128>, dim3(G), dim3(128), args, shm, st);
    return cudaLaunchCooperativeKernel((const void*)k_jacobi<256>, dim3(G), dim3(256), args, shm, st);
}

}  // namespace rutv
