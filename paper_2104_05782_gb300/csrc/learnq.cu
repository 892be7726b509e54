// learnq.cu -- the learned choice of the power-iteration count q (Sec. 3.2.1
// fixes q by hand; here a small network picks it per block step).
//
// Network: 16 features -> 64 -> 64 -> 4 logits, GELU after both hidden layers,
// softmax over q in {0, 1, 2, 3}; FP32.  Inputs are standardised with the
// (mu, sd) stored in the model.  Parameter layout (row-major, x W):
//   W1[16][64] b1[64] W2[64][64] b2[64] W3[64][4] b3[4] mu[16] sd[16]
// Features of block step i (written by k_learnq_features):
//   f[0..7]  = log10(|d_j| / |d_0|) of the previous block's d: the diagonal
//              of the R its panel QR produced (|R_jj| tracks the block's
//              singular values, and is ready before the block's b x b SVD, so
//              that SVD can overlap the next step) at j = 0, w/8, ..., 7w/8
//              (block 0: copies of f[8..15]);
//   f[9..15] = log10(|R_jj| / |R_00|) at j = w/8, ..., 7w/8, with R the
//              Householder R of the q = 0 sketch Y0 = T22^T G compressed to
//              at most 2b rows by a structured CountSketch (row r to row
//              r mod 2b with a random sign; Y0 itself when n' <= 2b),
//              factored in FP32 (b <= 128);
//   f[8]     = log10(||E||_F / ||E_0||_F), E that compressed sketch and E_0
//              the first block's: the level of the trailing matrix against
//              the whole (E[||S T22^T g||^2] = ||T22||_F^2 for a Gaussian g),
//              which tells a block of rounding noise (every choice of q is
//              as good) from a block inside a cluster of equal singular
//              values (flat ratios in both cases).
// Training kernels: per-sample forward, per-sample backward, gradient
// reductions over the batch in a fixed order (deterministic, no atomics),
// and Adam.  Cross-entropy loss averaged over the batch.
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr int NI = 16, NH = 64, NO = 4;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO, OFF_MU = OFF_B3 + NO, OFF_SD = OFF_MU + NI,
              NPARAM = OFF_SD + NI;
constexpr int NTRAIN = OFF_MU;  // trainable parameters (mu, sd are fixed)
constexpr float kLearnqConfidence = 0.999f;
// q = 0 is taken only for a block whose trailing matrix is below 1e-12 of the
// whole (f[8] <= -12): its singular values sit at the rounding level of any
// FP64 factorization of these sizes (n eps ||A|| ~ 1e-12 ||A|| at n = 16000).
// Above it the choice is at least 1: q = 0 inside a cluster of equal singular
// values leaves the cluster's directions in the trailing matrix at the size
// of the gap that follows (sigma_small / sigma_cluster, against its cube for
// q = 1), which distorts the blocks past the gap, while the training label
// looks at the block's own diagonal only.
constexpr float kLearnqNoiseLevel = -12.0f;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// forward of one sample; activations optional
__device__ void mlp_forward(const float* P, const float* xin, float* pre1, float* h1, float* pre2, float* h2,
                            float* logits) {
    float x[NI];
    for (int i = 0; i < NI; ++i) {
        float sd = P[OFF_SD + i];
        x[i] = (xin[i] - P[OFF_MU + i]) / (sd > 0.f ? sd : 1.f);
    }
    for (int j = 0; j < NH; ++j) {
        float s = P[OFF_B1 + j];
        for (int i = 0; i < NI; ++i) s = fmaf(x[i], P[OFF_W1 + i * NH + j], s);
        pre1[j] = s;
        h1[j] = gelu(s);
    }
    for (int j = 0; j < NH; ++j) {
        float s = P[OFF_B2 + j];
        for (int i = 0; i < NH; ++i) s = fmaf(h1[i], P[OFF_W2 + i * NH + j], s);
        pre2[j] = s;
        h2[j] = gelu(s);
    }
    for (int k = 0; k < NO; ++k) {
        float s = P[OFF_B3 + k];
        for (int i = 0; i < NH; ++i) s = fmaf(h2[i], P[OFF_W3 + i * NO + k], s);
        logits[k] = s;
    }
}

// Features of a block step (see the file comment).  R_jj are read from the
// QR storage of the compressed sketch (ld ldr); the previous block's d_j from
// dprev[j * dstride] (wprev = 0: first block of the call).  lvl[0] is the
// Frobenius norm of the compressed sketch when its caller computed it
// (have_level), else it is formed here from the upper triangle of the QR
// storage (the R factor has the same norm); lvl[1] keeps the first block's.
__global__ void k_learnq_features(const double* __restrict__ dprev, int64_t dstride, int wprev,
                                  const double* __restrict__ R, int64_t ldr, int w, float* __restrict__ f,
                                  double* __restrict__ lvl, int have_level) {
    const int t = threadIdx.x;
    __shared__ double s_level;
    if (t == 0) s_level = have_level ? lvl[0] : 0.0;
    if (!have_level) {  // one warp: column j of the upper triangle, fixed order
        double acc = 0.0;
        for (int j = t; j < w; j += 32)
            for (int i = 0; i <= j; ++i) {
                const double x = R[i + (int64_t)j * ldr];
                acc = fma(x, x, acc);
            }
        acc = warp_sum(acc);
        if (t == 0) s_level = sqrt(acc);
    }
    __syncwarp();
    if (t > 0 && t < 8) {
        int j = (t * w) / 8;
        double r0 = fabs(R[0]), rj = fabs(R[j + (int64_t)j * ldr]);
        float v = (r0 > 0.0 && rj > 0.0) ? (float)log10(rj / r0) : -16.0f;
        f[8 + t] = fmaxf(v, -16.0f);
    }
    if (t == 0) {
        const double level = s_level;
        if (wprev <= 0) lvl[1] = level;
        const double ref = (wprev <= 0) ? level : lvl[1];
        const float v = (level > 0.0 && ref > 0.0) ? (float)log10(level / ref) : -16.0f;
        f[8] = fmaxf(v, -16.0f);
    }
    __syncwarp();
    if (t < 8) {
        if (wprev <= 0) {
            f[t] = f[8 + t];
        } else {
            int j = (t * wprev) / 8;
            double d0 = fabs(dprev[0]), dj = fabs(dprev[(int64_t)j * dstride]);
            float v = (d0 > 0.0 && dj > 0.0) ? (float)log10(dj / d0) : -16.0f;
            f[t] = fmaxf(v, -16.0f);
        }
    }
}

// |R_jj| of the Householder QR of E (e x w, FP64, ld lde; e <= 256, w <= 128)
// for the learned-q features, in FP32 in one block of 32 warps.  E is held
// in registers: warp q owns columns q, q + 32, q + 64, q + 96 and lane l rows
// l, l + 32, ..., l + 224 of each.  E is scaled by a power of two (from its
// largest exponent) and cut to FP32 with integer instructions (truncation),
// so no FP64 instruction touches its 32768 entries.  Step j: the warp owning
// column j builds the reflector (dlarfg rule) from its registers and writes
// v to shared memory (two buffers by the parity of j, so one block barrier
// per step); every warp then applies it to its own columns right of j, with
// v read once per step.  Ratios |R_jj| / |R_00| come out to FP32 accuracy and
// saturate near 1e-7, where the remaining columns are rounding; the features
// clip there consistently in training and use.  *level = ||E||_F (an FP32
// sum of the scaled squares).
constexpr int FQR_THREADS = 1024;
constexpr int FQR_RP = 8;  // rows per lane (e <= 256)
constexpr int FQR_CP = 4;  // columns per warp (w <= 128)

// x 2^-s as FP32 by truncation, built from the FP64 bit pattern; values
// below the FP32 normal range give 0.
__device__ __forceinline__ float f64_to_f32_scaled(double x, int s) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((u >> 52) & 0x7FF);
    if (be == 0) return 0.0f;
    const int fe = be - 1023 - s + 127;
    if (fe <= 0) return 0.0f;
    const uint32_t bits = ((uint32_t)(u >> 63) << 31) | ((uint32_t)min(fe, 254) << 23) |
                          (uint32_t)((u >> 29) & 0x7FFFFFull);
    return __uint_as_float(bits);
}

__global__ void __launch_bounds__(FQR_THREADS) k_feature_rdiag32(const double* __restrict__ E, int64_t lde, int e, int w,
                                                                 double* __restrict__ rdiag, double* __restrict__ level) {
    __shared__ float vbuf[2][FQR_RP * 32];
    __shared__ float s_tau[2];
    __shared__ int s_be[32];
    __shared__ float s_ss[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the largest biased exponent of E (integer max of the bit patterns)
    int mbe = 0;
#pragma unroll
    for (int q = 0; q < FQR_CP; ++q) {
        const int c = warp + 32 * q;
#pragma unroll
        for (int k = 0; k < FQR_RP; ++k) {
            const int r = lane + 32 * k;
            if (c < w && r < e) {
                const unsigned long long u = (unsigned long long)__double_as_longlong(E[r + (int64_t)c * lde]);
                mbe = max(mbe, (int)((u >> 52) & 0x7FF));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) mbe = max(mbe, __shfl_xor_sync(0xffffffffu, mbe, o));
    if (lane == 0) s_be[warp] = mbe;
    __syncthreads();
    int gbe = 0;
    for (int k = 0; k < 32; ++k) gbe = max(gbe, s_be[k]);
    const int sc = (gbe == 0) ? 0 : gbe - 1023;  // |E| / 2^sc < 2
    float a[FQR_CP][FQR_RP];
    float ss = 0.0f;
#pragma unroll
    for (int q = 0; q < FQR_CP; ++q) {
        const int c = warp + 32 * q;
#pragma unroll
        for (int k = 0; k < FQR_RP; ++k) {
            const int r = lane + 32 * k;
            a[q][k] = (c < w && r < e) ? f64_to_f32_scaled(E[r + (int64_t)c * lde], sc) : 0.0f;
            ss = fmaf(a[q][k], a[q][k], ss);
        }
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) s_ss[warp] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < 32; ++k) t += s_ss[k];
        level[0] = ldexp(sqrt((double)t), sc);
    }
    const int steps = min(w, e);
    for (int j = 0; j < steps; ++j) {
        const int p = j & 1;
        const int qj = j >> 5;
        if (warp == (j & 31)) {  // the owner of column j builds its reflector
            float x[FQR_RP];
#pragma unroll
            for (int q = 0; q < FQR_CP; ++q)
                if (q == qj)
#pragma unroll
                    for (int k = 0; k < FQR_RP; ++k) x[k] = a[q][k];
            float xi2 = 0.0f;
#pragma unroll
            for (int k = 0; k < FQR_RP; ++k)
                if (lane + 32 * k > j) xi2 = fmaf(x[k], x[k], xi2);
            for (int o = 16; o > 0; o >>= 1) xi2 += __shfl_xor_sync(0xffffffffu, xi2, o);
            float alpha = 0.0f;
#pragma unroll
            for (int k = 0; k < FQR_RP; ++k)
                if (lane + 32 * k == j) alpha = x[k];
            alpha = __shfl_sync(0xffffffffu, alpha, j & 31);
            float beta = alpha, tau = 0.0f, inv = 0.0f;
            if (xi2 > 0.0f) {
                const float h = sqrtf(fmaf(alpha, alpha, xi2));
                beta = (alpha >= 0.0f) ? -h : h;
                tau = (beta - alpha) / beta;
                inv = 1.0f / (alpha - beta);
            }
#pragma unroll
            for (int k = 0; k < FQR_RP; ++k) {
                const int r = lane + 32 * k;
                const float v = (r > j) ? x[k] * inv : (r == j ? 1.0f : 0.0f);
                vbuf[p][r] = v;
                x[k] = (r > j) ? v : (r == j ? beta : x[k]);
            }
#pragma unroll
            for (int q = 0; q < FQR_CP; ++q)
                if (q == qj)
#pragma unroll
                    for (int k = 0; k < FQR_RP; ++k) a[q][k] = x[k];
            if (lane == 0) {
                rdiag[j] = fabs((double)beta);
                s_tau[p] = tau;
            }
        }
        __syncthreads();
        const float tau = s_tau[p];
        if (tau != 0.0f) {
            float v[FQR_RP];
#pragma unroll
            for (int k = 0; k < FQR_RP; ++k) v[k] = vbuf[p][lane + 32 * k];
#pragma unroll
            for (int q = 0; q < FQR_CP; ++q) {
                const int c = warp + 32 * q;
                if (c > j && c < w) {  // column c -= tau v (v^T column c), warp-uniform
                    float d = 0.0f;
#pragma unroll
                    for (int k = 0; k < FQR_RP; ++k) d = fmaf(v[k], a[q][k], d);
                    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                    d *= tau;
#pragma unroll
                    for (int k = 0; k < FQR_RP; ++k) a[q][k] = fmaf(-d, v[k], a[q][k]);
                }
            }
        }
    }
}

// E (e x w, ld e) = S Y (Y: L x w, ld ldy): the structured CountSketch
// that sends row r of Y to row r mod e of E with the sign of bit 0 of
// splitmix64(key + r) (Steele, Lea, Flood 2014).  One thread per entry of
// E sums its rows in order: deterministic, no atomics.  The loads of eight
// rows are issued before they are added, so that a thread waits for one
// memory round trip per eight rows rather than per row.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__global__ void k_countsketch(const double* __restrict__ Y, int64_t ldy, int64_t L, int w, int e, uint64_t key,
                              double* __restrict__ E) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)e * w) return;
    const int k = (int)(t % e), c = (int)(t / e);
    double s = 0.0;
    for (int64_t r0 = k; r0 < L; r0 += 8 * (int64_t)e) {
        double y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t r = r0 + u * (int64_t)e;
            y[u] = (r < L) ? Y[r + c * ldy] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t r = r0 + u * (int64_t)e;
            s += (splitmix64(key + (uint64_t)r) & 1ull) ? -y[u] : y[u];
        }
    }
    E[k + (int64_t)c * e] = s;
}

// The network predicts a distribution over the smallest adequate q.  The
// choice is risk-controlled: the smallest q whose cumulative predicted
// probability P(q_min <= q) reaches `confidence` (a plain argmax would accept
// every block the network is unsure about).  No model or a non-finite output
// gives `fallback`.
__global__ void __launch_bounds__(NH) k_learnq_infer(const float* __restrict__ P, const float* __restrict__ f,
                                                     int fallback, float confidence, int* q, int* qlog) {
    // one thread per hidden unit; each sum runs over the inputs in the same
    // order as mlp_forward
    __shared__ float x[NI], h1[NH], h2[NH], lg[NO];
    const int t = threadIdx.x;
    if (P == nullptr) {
        if (t == 0) {
            *q = fallback;
            if (qlog) *qlog = fallback;
        }
        return;
    }
    if (t < NI) {
        const float sd = P[OFF_SD + t];
        x[t] = (f[t] - P[OFF_MU + t]) / (sd > 0.f ? sd : 1.f);
    }
    __syncthreads();
    {
        float a = P[OFF_B1 + t];
        for (int i = 0; i < NI; ++i) a = fmaf(x[i], P[OFF_W1 + i * NH + t], a);
        h1[t] = gelu(a);
    }
    __syncthreads();
    {
        float a = P[OFF_B2 + t];
        for (int i = 0; i < NH; ++i) a = fmaf(h1[i], P[OFF_W2 + i * NH + t], a);
        h2[t] = gelu(a);
    }
    __syncthreads();
    if (t < NO) {
        float a = P[OFF_B3 + t];
        for (int i = 0; i < NH; ++i) a = fmaf(h2[i], P[OFF_W3 + i * NO + t], a);
        lg[t] = a;
    }
    __syncthreads();
    if (t != 0) return;
    bool finite = true;
    for (int k = 0; k < NO; ++k) finite &= isfinite(lg[k]);
    if (!finite) {
        *q = fallback;
        if (qlog) *qlog = fallback;
        return;
    }
    float mx = lg[0];
    for (int k = 1; k < NO; ++k) mx = fmaxf(mx, lg[k]);
    float pk[NO], se = 0.f;
    for (int k = 0; k < NO; ++k) {
        pk[k] = expf(lg[k] - mx);
        se += pk[k];
    }
    float cum = 0.f;
    int choice = NO - 1;
    for (int k = 0; k < NO; ++k) {
        cum += pk[k] / se;
        if (cum >= confidence) {
            choice = k;
            break;
        }
    }
    if (choice == 0 && !(f[8] <= kLearnqNoiseLevel)) choice = 1;
    *q = choice;
    if (qlog) *qlog = choice;
}

// per-sample forward + backward of the mean cross-entropy; writes the
// per-sample pieces the gradient reductions need.
__global__ void k_mlp_sample(const float* __restrict__ P, const float* __restrict__ X, const int* __restrict__ y,
                             int N, float* __restrict__ xs, float* __restrict__ h1s, float* __restrict__ h2s,
                             float* __restrict__ d1s, float* __restrict__ d2s, float* __restrict__ d3s,
                             float* __restrict__ loss, float* __restrict__ probs) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float pre1[NH], h1[NH], pre2[NH], h2[NH], lg[NO];
    const float* xin = X + (size_t)n * NI;
    mlp_forward(P, xin, pre1, h1, pre2, h2, lg);
    float mx = lg[0];
    for (int k = 1; k < NO; ++k) mx = fmaxf(mx, lg[k]);
    float pk[NO], se = 0.f;
    for (int k = 0; k < NO; ++k) {
        pk[k] = expf(lg[k] - mx);
        se += pk[k];
    }
    for (int k = 0; k < NO; ++k) pk[k] /= se;
    const int lab = y ? y[n] : 0;
    if (loss) loss[n] = -(lg[lab] - mx - logf(se));
    if (probs)
        for (int k = 0; k < NO; ++k) probs[(size_t)n * NO + k] = pk[k];
    if (!xs) return;
    const float invN = 1.0f / (float)N;
    float d3[NO];
    for (int k = 0; k < NO; ++k) d3[k] = (pk[k] - (k == lab ? 1.f : 0.f)) * invN;
    float d2[NH];
    for (int j = 0; j < NH; ++j) {
        float s = 0.f;
        for (int k = 0; k < NO; ++k) s = fmaf(d3[k], P[OFF_W3 + j * NO + k], s);
        d2[j] = s * gelu_d(pre2[j]);
    }
    float d1[NH];
    for (int j = 0; j < NH; ++j) {
        float s = 0.f;
        for (int k = 0; k < NH; ++k) s = fmaf(d2[k], P[OFF_W2 + j * NH + k], s);
        d1[j] = s * gelu_d(pre1[j]);
    }
    for (int i = 0; i < NI; ++i) {
        float sd = P[OFF_SD + i];
        xs[(size_t)n * NI + i] = (xin[i] - P[OFF_MU + i]) / (sd > 0.f ? sd : 1.f);
    }
    for (int j = 0; j < NH; ++j) {
        h1s[(size_t)n * NH + j] = h1[j];
        h2s[(size_t)n * NH + j] = h2[j];
        d1s[(size_t)n * NH + j] = d1[j];
        d2s[(size_t)n * NH + j] = d2[j];
    }
    for (int k = 0; k < NO; ++k) d3s[(size_t)n * NO + k] = d3[k];
}

// gradient entry g (of NTRAIN) = sum over samples in a fixed order
__global__ void k_mlp_grad(int N, const float* __restrict__ xs, const float* __restrict__ h1s,
                           const float* __restrict__ h2s, const float* __restrict__ d1s, const float* __restrict__ d2s,
                           const float* __restrict__ d3s, float* __restrict__ G) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NTRAIN) return;
    const float *a = nullptr, *d = nullptr;
    int na = 0, nd = 0, ia = 0, id = 0;
    if (g < OFF_B1) { int e = g - OFF_W1; a = xs; na = NI; ia = e / NH; d = d1s; nd = NH; id = e % NH; }
    else if (g < OFF_W2) { d = d1s; nd = NH; id = g - OFF_B1; }
    else if (g < OFF_B2) { int e = g - OFF_W2; a = h1s; na = NH; ia = e / NH; d = d2s; nd = NH; id = e % NH; }
    else if (g < OFF_W3) { d = d2s; nd = NH; id = g - OFF_B2; }
    else if (g < OFF_B3) { int e = g - OFF_W3; a = h2s; na = NH; ia = e / NO; d = d3s; nd = NO; id = e % NO; }
    else { d = d3s; nd = NO; id = g - OFF_B3; }
    float s = 0.f;
    for (int n = 0; n < N; ++n) {
        float dv = d[(size_t)n * nd + id];
        s = fmaf(a ? a[(size_t)n * na + ia] : 1.0f, dv, s);
    }
    G[g] = s;
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                       float* __restrict__ m2, int t, float lr, float wd) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NTRAIN) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float gr = G[g] + wd * P[g];
    m1[g] = b1 * m1[g] + (1.f - b1) * gr;
    m2[g] = b2 * m2[g] + (1.f - b2) * gr * gr;
    float mh = m1[g] / (1.f - powf(b1, (float)t));
    float vh = m2[g] / (1.f - powf(b2, (float)t));
    P[g] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_sum_loss(const float* __restrict__ l, int N, float* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += l[n];
    *out = (float)(s / (N > 0 ? N : 1));
}

}  // namespace

int learnq_nparam() { return NPARAM; }

cudaError_t countsketch(const double* Y, int64_t ldy, int64_t L, int w, int e, uint64_t key, double* E,
                        cudaStream_t st) {
    const int64_t total = (int64_t)e * w;
    if (total <= 0) return cudaSuccess;
    k_countsketch<<<(unsigned)cdiv(total, 128), 128, 0, st>>>(Y, ldy, L, w, e, key, E);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t feature_rdiag(const double* E, int64_t lde, int e, int w, double* rdiag, double* level,
                          cudaStream_t st) {
    if (e > 256 || w > 128 || e < 1 || w < 1) return cudaErrorInvalidValue;
    k_feature_rdiag32<<<1, FQR_THREADS, 0, st>>>(E, lde, e, w, rdiag, level);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t learnq_features(const double* dprev, int64_t dstride, int wprev, const double* R, int64_t ldr, int w,
                            float* f, double* lvl, bool have_level, cudaStream_t st) {
    k_learnq_features<<<1, 32, 0, st>>>(dprev, dstride, wprev, R, ldr, w, f, lvl, have_level ? 1 : 0);
    trace_count(1);
    return cudaGetLastError();
}

cudaError_t learnq_infer(const float* P, const float* f, int fallback, int* q, int* qlog, cudaStream_t st) {
    k_learnq_infer<<<1, NH, 0, st>>>(P, f, fallback, kLearnqConfidence, q, qlog);
    trace_count(1);
    return cudaGetLastError();
}

size_t learnq_train_scratch_floats(int N) { return (size_t)N * (NI + 4 * NH + NO + 1 + NO) + 4 * NPARAM + 8; }

// One step of (forward, backward[, Adam]) over the batch X (N x 16), labels y.
// grads: if non-null receives the gradient (NTRAIN floats); t > 0 applies Adam.
cudaError_t learnq_train_step(float* P, const float* X, const int* y, int N, float* scratch, float* grads_out,
                              float* loss_out, int t, float lr, float wd, cudaStream_t st) {
    float* xs = scratch;
    float* h1s = xs + (size_t)N * NI;
    float* h2s = h1s + (size_t)N * NH;
    float* d1s = h2s + (size_t)N * NH;
    float* d2s = d1s + (size_t)N * NH;
    float* d3s = d2s + (size_t)N * NH;
    float* loss = d3s + (size_t)N * NO;
    float* probs = loss + N;
    float* G = probs + (size_t)N * NO;
    float* m1 = G + NPARAM;
    float* m2 = m1 + NPARAM;
    k_mlp_sample<<<(N + 127) / 128, 128, 0, st>>>(P, X, y, N, xs, h1s, h2s, d1s, d2s, d3s, loss, nullptr);
    k_mlp_grad<<<(NTRAIN + 127) / 128, 128, 0, st>>>(N, xs, h1s, h2s, d1s, d2s, d3s, grads_out ? grads_out : G);
    trace_count(2);
    if (loss_out) {
        k_sum_loss<<<1, 32, 0, st>>>(loss, N, loss_out);
        trace_count(1);
    }
    if (t > 0) {
        k_adam<<<(NTRAIN + 127) / 128, 128, 0, st>>>(P, grads_out ? grads_out : G, m1, m2, t, lr, wd);
        trace_count(1);
    }
    return cudaGetLastError();
}

cudaError_t learnq_predict(const float* P, const float* X, int N, float* probs, cudaStream_t st) {
    k_mlp_sample<<<(N + 127) / 128, 128, 0, st>>>(P, X, nullptr, N, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                    nullptr, nullptr, probs);
    trace_count(1);
    return cudaGetLastError();
}

}  // namespace rutv
