// svd.cu -- SVD of the b x b diagonal block by one-sided (Hestenes) Jacobi.
//
// Sec. 3.2.3 diagonalises T22(1:b, 1:b) = U_svd D V_svd^T to build V_beta and
// U_beta; the paper names no SVD method.  One-sided Jacobi is used because it
// keeps relative accuracy for tiny singular values and has a fixed, parallel
// pair schedule.  A pair of columns (p, q) is rotated when
// |a_p^T a_q| > tol sqrt(|a_p|^2 |a_q|^2), tol = w 2^-53, by the rotation that
// makes them orthogonal (zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t).
// Sweeps stop when no pair is rotated (cap: max_sweeps, else ST_NOCONV);
// k_jacobi_cluster also stops after a sweep whose couplings and rotation
// angles were all tiny, when the next sweep would rotate nothing.
// Output is canonical: singular values descending (stable on ties), columns of
// Us = a_j / |a_j| (Gram-Schmidt completion for zero values), and each pair
// negated when the entry of largest modulus of Vs(:, j) (lowest index on
// ties) is negative.
//
// GB300 design: FP64 runs at ~7 GFLOP/s per SM, so a single block would need
// tens of milliseconds for b = 128.  The w/2 disjoint pairs of every round of
// a round-robin ("circle") ordering are spread over many SMs instead:
//   - k_jacobi_cluster (default): one thread-block cluster of 16 blocks (8
//     where 16 cannot be scheduled); A and V live in the blocks' shared
//     memory, one warp rotates one pair through distributed shared memory,
//     the hardware cluster barrier separates rounds;
//   - k_jacobi: w/2 blocks of one cooperative launch, one pair per block, A
//     and V in an L2-resident global scratch, a software grid barrier between
//     rounds (used when the cluster's shared memory is too small, and by the
//     allocation-free entry point).
// The pair order differs from a cyclic-by-rows sweep, which changes only
// rounding: the converged, canonical SVD is the same.
#include <cooperative_groups.h>

#include <mutex>
#include <unordered_map>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace cg = cooperative_groups;

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
                                               int max_sweeps, double tol, int dense,
                                               const double* __restrict__ V0, long long spin_limit) {
    __shared__ double red[3 * (NT / 32)];
    __shared__ int s_flag;
    const int tid = threadIdx.x, G = gridDim.x, cta = blockIdx.x;
    unsigned target = 0;

    // A := upper triangle of R (all of R when dense), V := V0 or I (ld w)
    for (int c = cta; c < w; c += G)
        for (int r = tid; r < w; r += NT) {
            A[r + (size_t)c * w] = (dense || r <= c) ? R[r + (int64_t)c * ldr] : 0.0;
            V[r + (size_t)c * w] = V0 ? V0[r + (size_t)c * w] : ((r == c) ? 1.0 : 0.0);
        }
    if (cta == 0 && tid < 3) rot[tid] = 0;
    if (!grid_sync(bar, target, status, spin_limit)) return;

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
            if (!grid_sync(bar, target, status, spin_limit)) return;
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


// ---------------------------------------------------------------------------
// Cluster variant: one thread-block cluster of G blocks (G = 16 or 8, set at
// launch).  Column c of the working copies A and V lives in the shared memory
// of block c / cols_per_block.  Each round, the lanes of one warp take one
// pair (p, q) of the circle ordering, the rows split over the lanes, and read
// and write the columns through distributed shared memory.  GB300's FP64
// unit retires about one warp instruction per 64 clocks per SM sub-partition,
// so the w/2 pairs of a round go to w/2 different warps (four per block, one
// per sub-partition), and the rotation takes one square root, one division
// and one reciprocal square root; the hardware cluster barrier separates
// rounds.
// Same schedule, test and canonical output as k_jacobi; the rotation is the
// same up to rounding: with d = beta - alpha and g = 2 gamma,
// t = sign(d / g) |g| / (|d| + sqrt(d^2 + g^2)) equals
// sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) for zeta = d / g.
constexpr int JC_THREADS = 128;
constexpr int JC_LPP = 32;  // lanes per pair
constexpr int JC_ROWS = 8;  // rows per lane: the cluster variant takes w <= 256

__global__ void __launch_bounds__(JC_THREADS)
    k_jacobi_cluster(const double* __restrict__ R, int64_t ldr, int w, int n2, int cpb, double* __restrict__ D,
                     double* __restrict__ Us, double* __restrict__ Vs, int* status, int max_sweeps, double tol,
                     int dense, const double* __restrict__ V0) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double jsm[];
    double* Aloc = jsm;                       // cpb columns x w
    double* Vloc = jsm + (size_t)cpb * w;     // cpb columns x w
    double* nrm = Vloc + (size_t)cpb * w;     // cpb norms
    __shared__ int s_flag;
    const int G = (int)cluster.num_blocks();
    const int me = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane & (JC_LPP - 1);
    const int PPW = 32 / JC_LPP;                     // pairs per warp
    const int NWALL = G * (JC_THREADS / 32);
    const int npairs = n2 / 2;
    const double tol2 = tol * tol;

    for (int lc = 0; lc < cpb; ++lc) {
        const int c = me * cpb + lc;
        for (int r = tid; r < w; r += JC_THREADS) {
            Aloc[(size_t)lc * w + r] = (c < w && (dense || r <= c)) ? R[r + (int64_t)c * ldr] : 0.0;
            Vloc[(size_t)lc * w + r] = (V0 && c < w) ? V0[r + (size_t)c * w] : ((r == c) ? 1.0 : 0.0);
        }
    }
    auto colA = [&](int c) -> double* {
        return cluster.map_shared_rank(Aloc, c / cpb) + (size_t)(c % cpb) * w;
    };
    auto colV = [&](int c) -> double* {
        return cluster.map_shared_rank(Vloc, c / cpb) + (size_t)(c % cpb) * w;
    };
    cluster.sync();

    bool converged = (w <= 1);
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        if (tid == 0) s_flag = 0;
        cluster.sync();
        for (int round = 0; round < n2 - 1; ++round) {
            // global warp index: warp 0 of every block first
            for (int gw = warp * G + me; gw * PPW < npairs; gw += NWALL) {
                const int k = gw * PPW + lane / JC_LPP;
                int p = 0, q = 0;
                bool act = k < npairs;
                if (act) {
                    p = circle_elem(k, round, n2);
                    q = circle_elem(n2 - 1 - k, round, n2);
                    if (p > q) { int t = p; p = q; q = t; }
                    act = q < w;
                }
                // both columns of A and V in registers (rows sub, sub + 32, ...),
                // all loads issued before the reductions
                double* ap = act ? colA(p) : nullptr;
                double* aq = act ? colA(q) : nullptr;
                double* vp = act ? colV(p) : nullptr;
                double* vq = act ? colV(q) : nullptr;
                double xr[JC_ROWS], yr[JC_ROWS], ur[JC_ROWS], zr[JC_ROWS];
#pragma unroll
                for (int i = 0; i < JC_ROWS; ++i) {
                    const int r = sub + JC_LPP * i;
                    const bool ok = act && r < w;
                    xr[i] = ok ? ap[r] : 0.0;
                    yr[i] = ok ? aq[r] : 0.0;
                    ur[i] = ok ? vp[r] : 0.0;
                    zr[i] = ok ? vq[r] : 0.0;
                }
                double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
                for (int i = 0; i < JC_ROWS; ++i) {
                    al = fma(xr[i], xr[i], al);
                    be = fma(yr[i], yr[i], be);
                    ga = fma(xr[i], yr[i], ga);
                }
#pragma unroll
                for (int o = JC_LPP / 2; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (!act) continue;
                // exponent fields: non-finite checks and range tests without FP64 compares
                const int eal = (int)(((unsigned long long)__double_as_longlong(al) >> 52) & 0x7FF);
                const int ebe = (int)(((unsigned long long)__double_as_longlong(be) >> 52) & 0x7FF);
                const int ega = (int)(((unsigned long long)__double_as_longlong(ga) >> 52) & 0x7FF);
                if (eal == 0x7FF || ebe == 0x7FF || ega == 0x7FF) {
                    if (sub == 0) atomicOr(status, ST_NONFINITE);
                    continue;
                }
                // |gamma| > tol sqrt(alpha beta), squared where that cannot under- or overflow
                bool rot, big = true;
                if (ega == 0) {
                    rot = false;
                } else if (eal + ebe > 2046 - 960 && eal + ebe < 2046 + 960) {
                    const double g2 = ga * ga, pr = al * be;
                    rot = g2 > tol2 * pr;
                    big = g2 > 1e-16 * pr;  // coupling above 1e-8
                } else {
                    rot = fabs(ga) > tol * sqrt(al) * sqrt(be);
                }
                if (!rot) continue;
                const double d = be - al, g = 2.0 * ga;
                // t from its FP32 value when d and g are within FP32's range
                // (decided on the exponent bits: no FP64 compares): the FP32
                // square root and division are cheap, and c = 1/sqrt(1+t^2),
                // s = c t in FP64 keep the rotation orthogonal to FP64
                // rounding; an angle off by ~1e-7 only leaves ~1e-7 of the
                // pair's coupling to a later sweep.
                const int ed = (int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FF);
                const int eg = (int)(((unsigned long long)__double_as_longlong(g) >> 52) & 0x7FF);
                double t;
                if (eg > 1023 - 60 && eg < 1023 + 60 && (ed == 0 || (ed > 1023 - 60 && ed < 1023 + 60))) {
                    const float df = (float)d, gf = (float)g;
                    const float sg = (df == 0.0f || ((df > 0.0f) == (gf > 0.0f))) ? 1.0f : -1.0f;
                    t = (double)(sg * fabsf(gf) / (fabsf(df) + sqrtf(fmaf(df, df, gf * gf))));
                } else {
                    const double zeta = d / g;
                    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                }
                const double cs = rsqrt(fma(t, t, 1.0));
                const double sn = cs * t;
                // a rotation by more than ~1e-7 rad (nearly equal columns
                // rotate by up to 45 degrees however small their coupling)
                // can re-couple earlier pairs: not a final sweep
                big = big || (int)(((unsigned long long)__double_as_longlong(t) >> 52) & 0x7FF) > 1023 - 24;
#pragma unroll
                for (int i = 0; i < JC_ROWS; ++i) {
                    const int r = sub + JC_LPP * i;
                    if (r < w) {
                        ap[r] = fma(-sn, yr[i], cs * xr[i]);
                        aq[r] = fma(sn, xr[i], cs * yr[i]);
                        vp[r] = fma(-sn, zr[i], cs * ur[i]);
                        vq[r] = fma(sn, ur[i], cs * zr[i]);
                    }
                }
                if (sub == 0) atomicOr((int*)&s_flag, big ? 3 : 1);
            }
            cluster.sync();
        }
        // converged after a sweep without rotations, or after one whose
        // couplings were all below 1e-8 and whose rotation angles were all
        // below ~1e-7: each later rotation then disturbs an earlier pair by
        // at most its angle times that pair's coupling (~1e-15), and the
        // FP32-derived angles leave at most ~1e-7 of a coupling behind, all
        // below the tolerance, so the next sweep would rotate nothing
        int any = 0;
        for (int b = 0; b < G; ++b) any |= *cluster.map_shared_rank(&s_flag, b);
        converged = (any & 2) == 0;
        cluster.sync();  // every block has read the flags before they are reset
    }
    if (!converged && me == 0 && tid == 0) atomicOr(status, ST_NOCONV);

    // ---- canonical output: each block writes its own columns ---------------
    for (int lc = warp; lc < cpb; lc += JC_THREADS / 32) {
        double s2 = 0.0;
        for (int r = lane; r < w; r += 32) s2 += Aloc[(size_t)lc * w + r] * Aloc[(size_t)lc * w + r];
        s2 = warp_sum(s2);
        if (lane == 0) nrm[lc] = sqrt(s2);
    }
    cluster.sync();
    for (int lc = warp; lc < cpb; lc += JC_THREADS / 32) {
        const int c = me * cpb + lc;
        if (c >= w) continue;
        const double v = nrm[lc];
        int rank = 0;
        for (int c2 = lane; c2 < w; c2 += 32) {
            const double u = *(cluster.map_shared_rank(nrm, c2 / cpb) + (c2 % cpb));
            rank += (u > v) || (u == v && c2 < c);
        }
        for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
        // canonical sign: largest |Vs| entry (lowest index on ties) positive
        double vmax = -1.0;
        int imax = 0;
        for (int r = lane; r < w; r += 32) {
            double a = fabs(Vloc[(size_t)lc * w + r]);
            if (a > vmax) { vmax = a; imax = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, vmax, o);
            int oi = __shfl_xor_sync(0xffffffffu, imax, o);
            if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
        }
        const double sg = (Vloc[(size_t)lc * w + imax] < 0.0) ? -1.0 : 1.0;
        if (lane == 0) D[rank] = v;
        for (int r = lane; r < w; r += 32) {
            Vs[r + (size_t)rank * w] = sg * Vloc[(size_t)lc * w + r];
            Us[r + (size_t)rank * w] = (v > 0.0) ? sg * Aloc[(size_t)lc * w + r] / v : 0.0;
        }
    }
    __threadfence();
    cluster.sync();
    // left vectors of zero singular values: Gram-Schmidt (twice) on unit
    // vectors, then the pair's canonical sign (block 0, rare)
    if (me == 0 && tid == 0) {
        for (int j = 0; j < w; ++j) {
            if (D[j] > 0.0) continue;
            double* u = Us + (size_t)j * w;
            for (int e = 0; e < w; ++e) {
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
}

// ---------------------------------------------------------------------------
// FP32 preconditioner: the same one-sided Jacobi in FP32 on one block (A and
// V in shared memory, one warp per pair, w <= 128), on R scaled by a power of
// two so that its largest entry is below 2.  Its V (orthogonal to about
// 1e-6) is written out as FP64; the caller re-orthogonalises it in FP64 and
// runs the FP64 Jacobi on R Q0 with V starting at Q0, which then needs a few
// sweeps instead of the eight to ten from scratch.  FP32 arithmetic runs at
// 64 times the FP64 rate on GB300, so these sweeps cost little.
constexpr int J32_THREADS = 1024;
__global__ void __launch_bounds__(J32_THREADS) k_jacobi32(const double* __restrict__ R, int64_t ldr, int w, int n2,
                                                         double* __restrict__ Q0, int max_sweeps, float tol) {
    extern __shared__ float j32[];
    float* A = j32;               // column c at c * w
    float* V = j32 + (size_t)w * w;
    __shared__ int s_rot, s_emax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NW = J32_THREADS / 32;
    if (tid == 0) s_emax = 0;
    __syncthreads();
    int em = 0;
    for (int e = tid; e < w * w; e += J32_THREADS) {
        const int r = e % w, c = e / w;
        if (r <= c)
            em = max(em, (int)(((unsigned long long)__double_as_longlong(R[r + (int64_t)c * ldr]) >> 52) & 0x7FF));
    }
    atomicMax(&s_emax, em);
    __syncthreads();
    // 2^(1023 - emax) as a double (exact; the largest entry lands in [1, 2))
    const int ex = 2046 - min(max(s_emax, 1), 2045);
    const double scale = __longlong_as_double((long long)ex << 52);
    for (int e = tid; e < w * w; e += J32_THREADS) {
        const int r = e % w, c = e / w;
        A[e] = (r <= c) ? (float)(R[r + (int64_t)c * ldr] * scale) : 0.0f;
        V[e] = (r == c) ? 1.0f : 0.0f;
    }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            // one warp per pair (rows lane, lane + 32, ...: conflict-free
            // shared-memory rows), both columns of A and V in registers
            for (int k = warp; k < n2 / 2; k += NW) {
                int p = circle_elem(k, round, n2);
                int q = circle_elem(n2 - 1 - k, round, n2);
                if (p > q) { int t = p; p = q; q = t; }
                if (q >= w) continue;
                float* ap = A + (size_t)p * w;
                float* aq = A + (size_t)q * w;
                float* vp = V + (size_t)p * w;
                float* vq = V + (size_t)q * w;
                float xr[4], yr[4], ur[4], zr[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = lane + 32 * i;
                    const bool ok = r < w;
                    xr[i] = ok ? ap[r] : 0.f;
                    yr[i] = ok ? aq[r] : 0.f;
                    ur[i] = ok ? vp[r] : 0.f;
                    zr[i] = ok ? vq[r] : 0.f;
                }
                float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    al = fmaf(xr[i], xr[i], al);
                    be = fmaf(yr[i], yr[i], be);
                    ga = fmaf(xr[i], yr[i], ga);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (!(fabsf(ga) > tol * sqrtf(al * be))) continue;  // also skips NaN
                // fast intrinsics: this sweep only preconditions the FP64 one
                const float d = be - al, g = 2.0f * ga;
                const float hyp = __fsqrt_rn(fmaf(d, d, g * g));
                const float sg = (d == 0.0f || ((d > 0.0f) == (g > 0.0f))) ? 1.0f : -1.0f;
                const float t = sg * __fdividef(fabsf(g), fabsf(d) + hyp);
                const float cs = rsqrtf(fmaf(t, t, 1.0f));
                const float sn = cs * t;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = lane + 32 * i;
                    if (r < w) {
                        ap[r] = cs * xr[i] - sn * yr[i];
                        aq[r] = sn * xr[i] + cs * yr[i];
                        vp[r] = cs * ur[i] - sn * zr[i];
                        vq[r] = sn * ur[i] + cs * zr[i];
                    }
                }
                if (lane == 0) s_rot = 1;
            }
            __syncthreads();
        }
        const int any = s_rot;
        __syncthreads();
        if (!any) break;
    }
    for (int e = tid; e < w * w; e += J32_THREADS) Q0[e] = (double)V[e];
}

__global__ void k_triu(const double* __restrict__ R, int64_t ldr, int w, double* __restrict__ U) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w * w; e += gridDim.x * blockDim.x) {
        const int r = e % w, c = e / w;
        U[e] = (r <= c) ? R[r + (int64_t)c * ldr] : 0.0;
    }
}

// Cluster size of k_jacobi_cluster per device: 16 until a launch of that
// size is refused, then 8, then 0 (the cooperative grid kernel).
std::mutex g_jc_mu;
std::unordered_map<int, int> g_jc_size;

int jacobi_cluster_blocks() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_jc_mu);
    auto it = g_jc_size.find(dev);
    if (it != g_jc_size.end()) return it->second;
    if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    g_jc_size[dev] = 16;
    return 16;
}

void jacobi_cluster_refused(int g) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_jc_mu);
    g_jc_size[dev] = (g > 8) ? 8 : 0;
}

}  // namespace

size_t jacobi_scratch_elems(int w) { return (size_t)2 * w * w; }

cudaError_t jacobi32_precondition(const double* R, int64_t ldr, int w, double* Q0, int max_sweeps, cudaStream_t st) {
    if (w <= 0) return cudaSuccess;
    if (w > 128) return cudaErrorInvalidValue;
    const size_t shm = sizeof(float) * (size_t)2 * w * w;
    static thread_local size_t configured = 0;
    if (shm > 48 * 1024 && shm > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_jacobi32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
        configured = shm;
    }
    const int n2 = w + (w & 1);
    k_jacobi32<<<1, J32_THREADS, shm, st>>>(R, ldr, w, n2, Q0, max_sweeps, (float)w * 5.9604645e-8f);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t triu_copy(const double* R, int64_t ldr, int w, double* U, cudaStream_t st) {
    if (w <= 0) return cudaSuccess;
    k_triu<<<(unsigned)std::min(cdiv((int64_t)w * w, 256), (int64_t)1024), 256, 0, st>>>(R, ldr, w, U);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t jacobi_svd(const double* R, int64_t ldr, int w, double* D, double* Us, double* Vs, double* scratch,
                       unsigned* bar, int* counters, int* status, int max_sweeps, cudaStream_t st,
                       bool allow_cluster, bool dense, const double* V0) {
    const int dn = dense ? 1 : 0;
    if (w <= 0) return cudaSuccess;
    int n2 = w + (w & 1);
    double tol = (double)w * 1.1102230246251565e-16;
    // cluster variant when A and V fit in the cluster's shared memory; a
    // cluster size the device refuses at launch is not tried again
    for (int gcl = jacobi_cluster_blocks(); allow_cluster && gcl > 0; gcl = jacobi_cluster_blocks()) {
        const int cpb = (n2 + gcl - 1) / gcl;
        const size_t shm_cluster = sizeof(double) * ((size_t)2 * cpb * w + cpb);
        if (shm_cluster > 200 * 1024 || w > JC_LPP * JC_ROWS) break;
        static thread_local size_t configured = 0;
        if (shm_cluster > 48 * 1024 && shm_cluster > configured) {
            cudaError_t e = cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)shm_cluster);
            if (e != cudaSuccess) return e;
            configured = shm_cluster;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)gcl);
        cfg.blockDim = dim3(JC_THREADS);
        cfg.dynamicSmemBytes = shm_cluster;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)gcl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e =
            cudaLaunchKernelEx(&cfg, k_jacobi_cluster, R, ldr, w, n2, cpb, D, Us, Vs, status, max_sweeps, tol, dn, V0);
        if (e == cudaSuccess) {
            trace_count(1);
            return cudaSuccess;
        }
        cudaGetLastError();  // a refused configuration leaves no sticky error
        jacobi_cluster_refused(gcl);
    }
    int G = std::max(1, n2 / 2);
    double* A = scratch;
    double* V = scratch + (size_t)w * w;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    size_t shm = sizeof(double) * (size_t)w;
    long long spin_limit = wait_limit();
    void* args[] = {(void*)&R,      (void*)&ldr,        (void*)&w,   (void*)&n2,  (void*)&A,
                    (void*)&V,      (void*)&D,          (void*)&Us,  (void*)&Vs,  (void*)&bar,
                    (void*)&counters, (void*)&status,   (void*)&max_sweeps, (void*)&tol, (void*)&dn,
                    (void*)&V0,     (void*)&spin_limit};
    trace_count(1);
    if (w <= 128)
        return cudaLaunchCooperativeKernel((const void*)k_jacobi<128>, dim3(G), dim3(128), args, shm, st);
    return cudaLaunchCooperativeKernel((const void*)k_jacobi<256>, dim3(G), dim3(256), args, shm, st);
}

}  // namespace rutv
