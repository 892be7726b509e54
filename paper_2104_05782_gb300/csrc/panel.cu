// panel.cu -- Householder QR of a tall panel and the compact-WY triangular factor.
//
// The QR of the sketch Y (n' x b, builds V_alpha, Sec. 3.2.1) and the QR of the
// panel T22(:, 1:b) (m' x b, builds U_alpha, Sec. 3.2.2) are the chains of b
// dependent reflectors that Sec. 4.1 calls the synchronisation points of the
// algorithm.  Each reflector follows LAPACK's dlarfg rule (Sec. 2.2 "HQR"):
//   alpha = P(j,j), x = P(j+1:, j), xi = |x|;  xi == 0 -> tau = 0;
//   else beta = -sign(alpha) hypot(alpha, xi), tau = (beta - alpha)/beta,
//        v = x / (alpha - beta), P(j,j) = beta,
// and H_j = I - tau [1; v][1; v]^T is applied to the columns right of j.
//
// GB300 design: one cooperative launch over up to one block per SM.  Block g
// owns a contiguous slab of rows, so every entry of the panel is read and
// written by one block only and stays in that SM's L1/L2 path.  Each column
// needs exactly ONE grid barrier: in the same pass that applies H_j to its
// rows, a block also forms its partial sums sum_r x_r^2 and sum_r x_r P(r,c)
// for the NEXT column (x = the next sub-column, c > j+1).  Those partials are
// all that is needed to build the next reflector and its row vector
// w_c = P(j,c) + (sum_r x_r P(r,c)) / (alpha - beta), so after the barrier
// every block reduces them itself, in the same fixed block order (the result
// is deterministic and identical in every block).  The row j values needed by
// all blocks travel through a small pivot buffer written by the block owning
// that row.  Partials and pivot rows are double-buffered by column parity.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr int PNT = 256;          // threads per block of the panel kernel
constexpr int kMaxChunk = 4096;   // rows per block (shared-memory bound)

// Cross-block sums.  GB300 retires one FP64 warp instruction per 64 clocks
// per sub-partition, so one lane summing all G partials of a column in a
// dependent chain would take G x 64 clocks.  Instead tpc lanes (a power of
// two, as many as the 256 threads allow for the columns left) each sum the
// g = lane (mod tpc) terms, and a shuffle tree combines them: a fixed order,
// so every block gets the same bits.  The partials of one column are
// contiguous (pc[g] for block g), so the tpc lanes of a column read
// consecutive words, and each lane issues its loads in batches of kBatch
// before adding, so that a batch costs one L2 round trip.
constexpr int kBatch = 20;
__device__ __forceinline__ double split_colsum(const double* __restrict__ pc, int G, bool active, int sub, int tpc) {
    double s = 0.0;
    if (active) {
        for (int g0 = sub; g0 < G; g0 += kBatch * tpc) {
            double t[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int g = g0 + u * tpc;
                t[u] = (g < G) ? __ldcg(pc + g) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) s += t[u];
        }
    }
    for (int o = tpc / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Largest panel width of the variant that also forms W, the Gram matrix and
// the triangular factor (one lane per column).
constexpr int kGramMaxW = 32;

// SLAB = true keeps the block's rows [r0, r0 + chunk) of the panel in shared
// memory for the whole factorization (one load, one store), column c at
// c * ldp with ldp = 1 (mod 16) so that lanes walking along a row hit
// distinct banks; false works on the panel in global memory.
//
// GRAM = true (w <= kGramMaxW) also produces the compact WY form of the
// panel (Sec. 2.3) in the same launch: W (len x w, ld len, unit lower
// trapezoidal), the Gram matrix W^T W and Tf.  Entry (i, j), i < j, of the
// Gram matrix is w_i(j) + sum_{r > j} w_i(r) w_j(r); its block partial is
// formed in the pass that applies H_j, by the lanes i < j that would
// otherwise idle there (the lanes right of j update the panel), so it adds
// no FP64 instruction to that pass.  After the last column two more grid
// barriers: block b reduces Gram column b, then block b forms column b of
// Tf by the back substitution of k_tfactor_col.
template <bool SLAB, bool GRAM>
__global__ void __launch_bounds__(PNT) k_panel_qr(double* __restrict__ P, int64_t ld, int len, int w,
                                                  double* __restrict__ tau, double* __restrict__ part_d,
                                                  double* __restrict__ piv, unsigned* bar, int* status,
                                                  int chunk, int ldp, long long spin_limit,
                                                  double* __restrict__ Wout, double* __restrict__ Tf,
                                                  double* __restrict__ gpart, double* __restrict__ gred) {
    extern __shared__ double smem[];
    constexpr int NW = PNT / 32;
    double* xsb0 = smem;
    double* xsb1 = smem + chunk;
    double* sred = smem + 2 * chunk;
    double* wv = sred + w;
    double* pivs = wv + w;         // pivot row j of the current column, columns j..w-1
    double* wred = pivs + w;       // NW x w: per-warp partial dot products
    double* slab = wred + NW * w;  // ldp x w (SLAB only)
    double* part = part_d;         // [parity][column][block]
    __shared__ double s_scalars[5];

    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = cta * chunk;
    const int r1 = min(len, r0 + chunk);
    const int nr = max(0, r1 - r0);
    const int RB = (nr + NW - 1) / NW;  // rows per warp in the column-parallel passes
    const int t0 = min(nr, warp * RB), t1 = min(nr, t0 + RB);
    unsigned target = 0;
    // entry (r0 + t, c) of the panel, t < nr: own rows only
    auto PX = [&](int t, int c) -> double& {
        return SLAB ? slab[t + (size_t)c * ldp] : P[(r0 + t) + (int64_t)c * ld];
    };
    if (SLAB) {
        for (int c = warp; c < w; c += NW)
            for (int t = lane; t < nr; t += 32) slab[t + (size_t)c * ldp] = P[(r0 + t) + (int64_t)c * ld];
        __syncthreads();
    }

    // ---- prologue: partials of column 0 ------------------------------------
    for (int t = tid; t < nr; t += PNT) {
        int r = r0 + t;
        xsb0[t] = (r > 0) ? PX(t, 0) : 0.0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < w; c0 += 32) {  // lanes over columns, warps over rows
        const int c = c0 + lane;
        if (c < w) {
            double acc = 0.0;
            for (int t = t0; t < t1; ++t) acc = fma(xsb0[t], c == 0 ? xsb0[t] : PX(t, c), acc);
            wred[warp * w + c] = acc;
        }
    }
    __syncthreads();
    for (int c = tid; c < w; c += PNT) {
        double acc = wred[c];
        for (int k = 1; k < NW; ++k) acc += wred[k * w + c];
        part[(size_t)c * G + cta] = acc;
    }
    if (r0 <= 0 && 0 < r1)
        for (int c = tid; c < w; c += PNT) piv[c] = PX(0, c);
    if (!grid_sync(bar, target, status, spin_limit)) return;

    for (int j = 0; j < w; ++j) {
        const int p = j & 1;
        double* xc = p ? xsb1 : xsb0;
        double* xn = p ? xsb0 : xsb1;
        const double* pp = part + (size_t)p * G * w;
        const double* pv = piv + (size_t)p * w;

        // the pivot row and the partials of columns j..w-1 are read in one
        // round: tpc lanes per column reduce the partials
        for (int c = j + tid; c < w; c += PNT) pivs[c] = __ldcg(pv + c);
        {
            int tpc = 1;
            while (tpc < 32 && tpc * 2 * (w - j) <= PNT) tpc *= 2;
            const int cpp = PNT / tpc;  // columns per pass
            for (int c0 = j; c0 < w; c0 += cpp) {
                const int c = c0 + tid / tpc;
                const double v = split_colsum(pp + (size_t)c * G, G, c < w, tid & (tpc - 1), tpc);
                if (c < w && (tid & (tpc - 1)) == 0) sred[c] = v;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double alpha = pivs[j];
            double xi2 = sred[j];
            double tj = 0.0, beta = alpha, d = 1.0, act = 0.0, rd = 1.0;
            if (!isfinite(xi2) || !isfinite(alpha)) {
                atomicOr(status, ST_NONFINITE);
            } else if (xi2 > 0.0) {
                const double h = (fabs(alpha) < 1e150 && xi2 < 1e300) ? sqrt(fma(alpha, alpha, xi2))
                                                                        : hypot(alpha, sqrt(xi2));
                beta = (alpha >= 0.0) ? -h : h;
                tj = (beta - alpha) / beta;
                d = alpha - beta;
                rd = 1.0 / d;
                act = 1.0;
            }
            s_scalars[0] = tj;
            s_scalars[1] = beta;
            s_scalars[2] = d;
            s_scalars[3] = act;
            s_scalars[4] = rd;
            if (cta == 0) tau[j] = tj;
        }
        __syncthreads();
        const double tj = s_scalars[0], beta = s_scalars[1], rd = s_scalars[4];
        const bool act = s_scalars[3] != 0.0;
        for (int c = j + 1 + tid; c < w; c += PNT) wv[c] = act ? fma(sred[c], rd, pivs[c]) : 0.0;

        // (a) v_r = x_r / d on own rows r > j; P(j,j) = beta; xc keeps tau_j v_r
        if (act) {
            for (int t = tid; t < nr; t += PNT) {
                int r = r0 + t;
                if (r > j) {
                    double v = xc[t] * rd;
                    xc[t] = tj * v;
                    PX(t, j) = v;
                }
            }
            if (tid == 0 && r0 <= j && j < r1) PX(j - r0, j) = beta;
        }
        __syncthreads();
        if (j + 1 >= w) break;

        // (b1) column j+1 on own rows r > j; next sub-column x' (rows > j+1); row j
        for (int t = tid; t < nr; t += PNT) {
            int r = r0 + t;
            double val = 0.0;
            if (r > j) {
                double* e = &PX(t, j + 1);
                val = *e;
                if (act) {
                    val = fma(-xc[t], wv[j + 1], val);
                    *e = val;
                }
            }
            xn[t] = (r > j + 1) ? val : 0.0;
        }
        if (act && r0 <= j && j < r1)
            for (int c = j + 1 + tid; c < w; c += PNT) PX(j - r0, c) = pivs[c] - tj * wv[c];
        __syncthreads();

        // (b2) on rows t0..t1 of this warp, lanes over columns c:
        //   c >= j+2: apply H_j, then the next column's partial sum_r x'_r P(r,c);
        //   c == j+1: sum_r x'_r^2 (x' is column j+1 below row j+1, already updated);
        //   c < j (GRAM): the Gram partial sum_{r > j} w_c(r) w_j(r).
        for (int c0 = GRAM ? 0 : j + 1; c0 < w; c0 += 32) {
            const int c = c0 + lane;
            if (c < w && c != j) {
                const bool apply = act && c > j + 1;
                const double wc = apply ? wv[c] : 0.0;
                double acc = 0.0;
                for (int t = t0; t < t1; ++t) {
                    if (r0 + t > j) {
                        double* e = &PX(t, c);
                        double val = *e;
                        if (apply) {
                            val = fma(-xc[t], wc, val);
                            *e = val;
                        }
                        acc = fma(c > j ? xn[t] : PX(t, j), val, acc);
                    }
                }
                wred[warp * w + c] = acc;
            }
        }
        __syncthreads();
        for (int c = j + 1 + tid; c < w; c += PNT) {
            double acc = wred[c];
            for (int k = 1; k < NW; ++k) acc += wred[k * w + c];
            part[(size_t)(p ^ 1) * G * w + (size_t)c * G + cta] = acc;
        }
        if (GRAM)
            for (int c = tid; c < j; c += PNT) {
                double acc = wred[c];
                for (int k = 1; k < NW; ++k) acc += wred[k * w + c];
                if (r0 <= j && j < r1) acc += PX(j - r0, c);  // w_j(j) = 1
                gpart[((size_t)j * w + c) * G + cta] = acc;
            }
        if (r0 <= j + 1 && j + 1 < r1)
            for (int c = j + 1 + tid; c < w; c += PNT)
                piv[(size_t)(p ^ 1) * w + c] = PX(j + 1 - r0, c);
        if (!grid_sync(bar, target, status, spin_limit)) return;
    }
    if (GRAM && w > 1) {  // Gram column w-1 (its reflector came last)
        const int j = w - 1;
        if (lane < j) {
            double acc = 0.0;
            for (int t = t0; t < t1; ++t)
                if (r0 + t > j) acc = fma(PX(t, j), PX(t, lane), acc);
            wred[warp * w + lane] = acc;
        }
        __syncthreads();
        for (int c = tid; c < j; c += PNT) {
            double acc = wred[c];
            for (int k = 1; k < NW; ++k) acc += wred[k * w + c];
            if (r0 <= j && j < r1) acc += PX(j - r0, c);
            gpart[((size_t)j * w + c) * G + cta] = acc;
        }
    }
    if (GRAM) {  // W on own rows
        for (int c = warp; c < w; c += NW)
            for (int t = lane; t < nr; t += 32) {
                const int r = r0 + t;
                Wout[r + (int64_t)c * len] = (r < c) ? 0.0 : (r == c ? 1.0 : PX(t, c));
            }
    }
    if (SLAB) {
        __syncthreads();
        for (int c = warp; c < w; c += NW)
            for (int t = lane; t < nr; t += 32) P[(r0 + t) + (int64_t)c * ld] = slab[t + (size_t)c * ldp];
    }
    if (GRAM) {
        if (!grid_sync(bar, target, status, spin_limit)) return;
        // block b: Gram column b, entries i < b (warps over i, lanes over blocks)
        for (int b = cta; b < w; b += G)
            for (int i = warp; i < b; i += NW) {
                const double* src = gpart + ((size_t)b * w + i) * G;
                double sacc = 0.0;
                for (int g0 = lane; g0 < G; g0 += 32 * 8) {
                    double t8[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) t8[u] = (g0 + 32 * u < G) ? __ldcg(src + g0 + 32 * u) : 0.0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) sacc += t8[u];
                }
                sacc = warp_sum(sacc);
                if (lane == 0) gred[i + (size_t)b * w] = sacc;
            }
        if (!grid_sync(bar, target, status, spin_limit)) return;
        // block b: column b of Tf (as k_tfactor_col), the triangle of Gram
        // columns 1..b staged in shared memory after the slab
        double* gs = slab + (SLAB ? (size_t)ldp * w : 0);  // packed triangle
        double* tacc = gs + kGramMaxW * (kGramMaxW - 1) / 2;
        for (int b = cta; b < w; b += G) {
            __syncthreads();
            for (int e = tid; e < b * kGramMaxW; e += PNT) {
                const int k = e / kGramMaxW, i = e % kGramMaxW;  // column k + 1, row i
                if (i < k + 1) gs[(k + 1) * k / 2 + i] = __ldcg(gred + i + (size_t)(k + 1) * w);
            }
            for (int i = tid; i < b; i += PNT) tacc[i] = 0.0;
            __syncthreads();
            if (warp == 0) {
                double* x = Tf + (size_t)b * w;
                for (int i = b + 1 + lane; i < w; i += 32) x[i] = 0.0;
                const double tb = __ldcg(tau + b);
                if (lane == 0) {
                    if (!isfinite(tb)) atomicOr(status, ST_NONFINITE);
                    x[b] = tb;
                }
                double xk = tb;
                for (int k = b; k >= 1; --k) {
                    if (lane < k) tacc[lane] = fma(gs[k * (k - 1) / 2 + lane], xk, tacc[lane]);
                    __syncwarp();
                    xk = -__ldcg(tau + k - 1) * tacc[k - 1];
                    if (lane == 0) x[k - 1] = xk;
                }
            }
        }
    }
}

__global__ void k_extract_w(const double* __restrict__ P, int64_t ld, int len, int w, double* __restrict__ W) {
    int64_t total = (int64_t)len * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % len);
        int c = (int)(e / len);
        W[e] = (r < c) ? 0.0 : (r == c ? 1.0 : P[r + (int64_t)c * ld]);
    }
}

// Triangular factor of the compact WY form (Sec. 2.3): Q = H_0 ... H_{w-1} =
// I - W Tf W^T.  Tf is the inverse of S = diag(1 / tau) + strict_upper(W^T W)
// (the column recurrence Tf(0:j, j) = -tau_j Tf(0:j,0:j) (W^T W)(0:j, j)
// written as one triangular solve per column), so every column is an
// independent back substitution:
//   Tf(j, j) = tau_j,  Tf(i, j) = -tau_i sum_{k=i+1..j} (W^T W)(i, k) Tf(k, j),
// which also holds for tau_i = 0 (H_i = I gives a zero row and column).
// One thread per column; the Gram matrix is staged in shared memory when it
// fits.
__global__ void k_tfactor(const double* __restrict__ gram, const double* __restrict__ tau, int w,
                          double* __restrict__ Tf, int use_smem, int* status) {
    extern __shared__ double gsm[];
    const double* G = gram;
    if (use_smem) {
        for (int e = threadIdx.x; e < w * w; e += blockDim.x) gsm[e] = gram[e];
        __syncthreads();
        G = gsm;
    }
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
        double* x = Tf + (size_t)j * w;
        for (int i = j + 1; i < w; ++i) x[i] = 0.0;
        const double tj = tau[j];
        if (!isfinite(tj)) atomicOr(status, ST_NONFINITE);
        x[j] = tj;
        for (int i = j - 1; i >= 0; --i) {
            double s0 = 0.0, s1 = 0.0;
            int k = i + 1;
            for (; k + 1 <= j; k += 2) {
                s0 += G[i + (size_t)k * w] * x[k];
                s1 += G[i + (size_t)(k + 1) * w] * x[k + 1];
            }
            if (k <= j) s0 += G[i + (size_t)k * w] * x[k];
            x[i] = -tau[i] * (s0 + s1);
        }
    }
}

// Same triangular factor, one block per column j and the substitution
// written column-oriented: once Tf(k, j) is known, lane i adds
// (W^T W)(i, k) Tf(k, j) to its running sum for every row i < k, and
// Tf(k-1, j) = -tau_{k-1} sum(k-1) is then complete.  Every step is one FMA
// per lane and a warp-level exchange, so the w-long dependent chain costs
// about w short steps instead of w dot products; warp 0 runs it.  STAGED
// (w <= 128): first all TF_THREADS threads copy the block's triangle of the
// Gram matrix into shared memory, packed (column k, rows 0..k-1, at offset
// k (k - 1) / 2), each warp with several columns' loads in flight, so that
// the copy costs a few L2 round trips rather than one per column; otherwise
// (w <= 256) warp 0 reads the L2-resident Gram matrix itself.
constexpr int TF_MAXW = 256;
constexpr int TF_STAGEW = 128;
constexpr int TF_THREADS = 256;
template <bool STAGED>
__global__ void __launch_bounds__(TF_THREADS) k_tfactor_col(const double* __restrict__ gram,
                                                            const double* __restrict__ tau, int w,
                                                            double* __restrict__ Tf, int* status) {
    extern __shared__ double gs[];
    __shared__ double acc[TF_MAXW];
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto G = [&](int i, int k) -> double { return STAGED ? gs[k * (k - 1) / 2 + i] : __ldg(gram + i + (size_t)k * w); };
    if (STAGED) {
        constexpr int NWARP = TF_THREADS / 32, U = 4, Q = TF_STAGEW / 32;
        for (int k0 = 1 + warp; k0 <= j; k0 += U * NWARP) {
            double t[U][Q];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = k0 + u * NWARP;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int i = lane + 32 * q;
                    t[u][q] = (k <= j && i < k) ? __ldg(gram + i + (size_t)k * w) : 0.0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = k0 + u * NWARP;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int i = lane + 32 * q;
                    if (k <= j && i < k) gs[k * (k - 1) / 2 + i] = t[u][q];
                }
            }
        }
        __syncthreads();
    }
    if (warp != 0) return;
    for (int i = lane; i < j; i += 32) acc[i] = 0.0;
    double* x = Tf + (size_t)j * w;
    for (int i = j + 1 + lane; i < w; i += 32) x[i] = 0.0;
    const double tj = tau[j];
    if (lane == 0) {
        if (!isfinite(tj)) atomicOr(status, ST_NONFINITE);
        x[j] = tj;
    }
    __syncwarp();
    double xk = tj;
    for (int k = j; k >= 1; --k) {
        for (int i = lane; i < k; i += 32) acc[i] = fma(G(i, k), xk, acc[i]);
        __syncwarp();
        xk = -tau[k - 1] * acc[k - 1];
        if (lane == 0) x[k - 1] = xk;
    }
}

}  // namespace

int panel_qr_grid(int64_t len, int w, int sms) {
    (void)w;
    int64_t g = cdiv(len, 64);
    if (g > sms) g = sms;
    if (g < 1) g = 1;
    while (cdiv(len, g) > kMaxChunk) ++g;  // only for len > sms * kMaxChunk
    return (int)g;
}

size_t panel_qr_scratch_elems(int w, int grid) {
    const size_t g = (size_t)std::min(w, kGramMaxW);
    return (size_t)2 * grid * w + (size_t)2 * w + g * g * ((size_t)grid + 1);
}

namespace {

// Shared by panel_qr and panel_qr_wy; W == nullptr selects the plain variant.
cudaError_t panel_qr_launch(double* P, int64_t ld, int64_t len, int w, double* tau, double* W, double* Tf,
                            double* scratch, unsigned* bar, int* status, int sms, cudaStream_t st) {
    if (len <= 0 || w <= 0) return cudaSuccess;
    const bool gram = W != nullptr;
    if (gram && w > kGramMaxW) return cudaErrorInvalidValue;
    int G = panel_qr_grid(len, w, sms);
    int chunk = (int)cdiv(len, G);
    if (chunk > kMaxChunk || G > sms) return cudaErrorInvalidValue;
    double* part = scratch;
    double* piv = scratch + (size_t)2 * G * w;
    double* gpart = piv + (size_t)2 * w;
    double* gred = gpart + (size_t)w * w * G;
    const int ldp = chunk + ((17 - chunk % 16) % 16);  // = 1 (mod 16)
    const size_t base = sizeof(double) * ((size_t)2 * chunk + (size_t)3 * w + (size_t)(PNT / 32) * w);
    const size_t tail = gram ? sizeof(double) * (size_t)(kGramMaxW * (kGramMaxW - 1) / 2 + kGramMaxW) : 0;
    const size_t with_slab = base + sizeof(double) * (size_t)ldp * w + tail;
    const bool use_slab = with_slab <= 220 * 1024;
    const size_t shm = use_slab ? with_slab : base + tail;
    const void* fns[4] = {(const void*)k_panel_qr<false, false>, (const void*)k_panel_qr<true, false>,
                          (const void*)k_panel_qr<false, true>, (const void*)k_panel_qr<true, true>};
    const int which = (use_slab ? 1 : 0) + (gram ? 2 : 0);
    static thread_local size_t configured[4] = {0, 0, 0, 0};
    if (shm > 48 * 1024 && shm > configured[which]) {
        cudaError_t e = cudaFuncSetAttribute(fns[which], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
        configured[which] = shm;
    }
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int len_i = (int)len;
    int ldp_i = ldp;
    long long spin_limit = wait_limit();
    void* args[] = {&P,     &ld,   &len_i, &w,          &tau, &part, &piv,  &bar,
                    &status, &chunk, &ldp_i, &spin_limit, &W,   &Tf,   &gpart, &gred};
    trace_count(1);
    return cudaLaunchCooperativeKernel(fns[which], dim3(G), dim3(PNT), args, shm, st);
}

}  // namespace

cudaError_t panel_qr(double* P, int64_t ld, int64_t len, int w, double* tau, double* scratch, unsigned* bar,
                     int* status, int sms, cudaStream_t st) {
    return panel_qr_launch(P, ld, len, w, tau, nullptr, nullptr, scratch, bar, status, sms, st);
}

cudaError_t panel_qr_wy(double* P, int64_t ld, int64_t len, int w, double* tau, double* W, double* Tf,
                        double* scratch, unsigned* bar, int* status, int sms, cudaStream_t st) {
    if (W == nullptr || Tf == nullptr) return cudaErrorInvalidValue;
    return panel_qr_launch(P, ld, len, w, tau, W, Tf, scratch, bar, status, sms, st);
}

cudaError_t extract_w(const double* P, int64_t ld, int64_t len, int w, double* W, cudaStream_t st) {
    if (len <= 0 || w <= 0) return cudaSuccess;
    int64_t total = len * w;
    unsigned blocks = (unsigned)std::min<int64_t>(cdiv(total, 256), 4096);
    k_extract_w<<<blocks, 256, 0, st>>>(P, ld, (int)len, w, W);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t tfactor(const double* gram, const double* tau, int w, double* Tf, int* status, cudaStream_t st) {
    if (w <= 0) return cudaSuccess;
    const size_t bytes = sizeof(double) * (size_t)w * w;
    const int use_smem = bytes <= 200 * 1024;
    const size_t shm = use_smem ? bytes : 0;
    static thread_local size_t configured = 0;
    if (shm > 48 * 1024 && shm > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tfactor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
        configured = shm;
    }
    if (w <= TF_STAGEW) {
        const size_t tri = sizeof(double) * (size_t)w * (w - 1) / 2;
        static thread_local size_t configured_col = 0;
        if (tri > 48 * 1024 && tri > configured_col) {
            cudaError_t e =
                cudaFuncSetAttribute(k_tfactor_col<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tri);
            if (e != cudaSuccess) return e;
            configured_col = tri;
        }
        k_tfactor_col<true><<<w, TF_THREADS, tri, st>>>(gram, tau, w, Tf, status);
        trace_count(1);
        return cudaGetLastError();
    }
    if (w <= TF_MAXW) {
        k_tfactor_col<false><<<w, TF_THREADS, 0, st>>>(gram, tau, w, Tf, status);
        trace_count(1);
        return cudaGetLastError();
    }
    const int threads = std::min(1024, ((w + 31) / 32) * 32);
    k_tfactor<<<1, threads, shm, st>>>(gram, tau, w, Tf, use_smem, status);
    trace_count(1);
    return cudaGetLastError();
}

}  // namespace rutv
