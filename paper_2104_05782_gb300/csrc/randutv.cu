// randutv.cu -- host driver and exported C ABI of librandutv (declared in
// include/randutv.h).
//
// The block step follows the outline of Sec. 3.2 and the Householder /
// compact-WY form of the FLAME algorithm of Sec. 4.3, with every arithmetic
// operation in a kernel of this library:
//   sketch  (Sec. 3.2.1): G Gaussian, Y = T22^T G, q x { Z = T22 Y, Y = T22^T Z }
//   V_alpha (Sec. 3.2.1): Householder QR of Y -> W_V, tau_V, Tf_V
//                         T(:, J2) -= (T(:, J2) W_V) Tf_V W_V^T over ALL m rows
//                         (Sec. 5.4: the right application covers every row),
//                         V(:, J2) likewise
//   U_alpha (Sec. 3.2.2): Householder QR of T22(:, 1:b) -> W_U, tau_U, Tf_U
//                         T22(:, b+1:) -= W_U Tf_U^T (W_U^T T22(:, b+1:))
//                         U(:, I2) -= (U(:, I2) W_U) Tf_U W_U^T
//   SVD     (Sec. 3.2.3): R = Us D Vs^T; T(blk,blk) = D; T(0:k0, blk) *= Vs;
//                         T(blk, rest) = Us^T T(blk, rest); V(:,blk) *= Vs;
//                         U(:,blk) *= Us; T below the block := 0.
// When at most b columns remain, the trailing block gets the panel QR and the
// SVD without a sketch (the Matlab listing of Sec. 3.2 takes a full SVD there).
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/randutv.h"
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxSweeps = 30;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Workspace {
    double *G, *Y, *Z, *W, *X, *X2, *tmp, *part, *tau, *Tf, *gram, *pscr, *jscr, *D, *Us, *Vs;
    unsigned* bars;
    int* counters;
    int* status;
    size_t part_elems;
};

struct Layout {
    size_t off[20];
    size_t total;
    size_t part_elems;
};

int device_sms(int dev) {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    cache[dev] = sms;
    return sms;
}

Layout make_layout(int64_t m, int64_t n, int b, int sms) {
    Layout L{};
    int64_t mx = std::max<int64_t>(std::max(m, n), 1);
    int64_t bb = std::max(b, 1);
    int64_t wmax = std::min<int64_t>(bb, std::max<int64_t>(n, 1));
    size_t part = (size_t)8 * sms * 64 * 64 + (size_t)2 * mx * wmax;
    size_t sizes[20] = {
        sizeof(double) * (size_t)mx * wmax,          // G
        sizeof(double) * (size_t)mx * wmax,          // Y
        sizeof(double) * (size_t)mx * wmax,          // Z
        sizeof(double) * (size_t)mx * wmax,          // W
        sizeof(double) * (size_t)mx * wmax,          // X
        sizeof(double) * (size_t)mx * wmax,          // X2
        sizeof(double) * (size_t)mx * wmax,          // tmp
        sizeof(double) * part,                       // split-K partials
        sizeof(double) * (size_t)wmax,               // tau
        sizeof(double) * (size_t)2 * wmax * wmax,    // Tf (+ row-major scratch)
        sizeof(double) * (size_t)wmax * wmax,        // gram
        sizeof(double) * panel_qr_scratch_elems((int)wmax, sms + 8),
        sizeof(double) * jacobi_scratch_elems((int)wmax),
        sizeof(double) * (size_t)wmax,               // D
        sizeof(double) * (size_t)wmax * wmax,        // Us
        sizeof(double) * (size_t)wmax * wmax,        // Vs
        sizeof(unsigned) * 64,                       // barrier counters
        sizeof(int) * 64,                            // Jacobi rotation counters
        sizeof(int) * 64,                            // status word
        0};
    size_t o = 0;
    for (int i = 0; i < 20; ++i) {
        L.off[i] = o;
        o += align_up(sizes[i]);
    }
    L.total = o;
    L.part_elems = part;
    return L;
}

Workspace carve(void* base, const Layout& L) {
    char* p = (char*)base;
    Workspace w{};
    w.G = (double*)(p + L.off[0]);
    w.Y = (double*)(p + L.off[1]);
    w.Z = (double*)(p + L.off[2]);
    w.W = (double*)(p + L.off[3]);
    w.X = (double*)(p + L.off[4]);
    w.X2 = (double*)(p + L.off[5]);
    w.tmp = (double*)(p + L.off[6]);
    w.part = (double*)(p + L.off[7]);
    w.tau = (double*)(p + L.off[8]);
    w.Tf = (double*)(p + L.off[9]);
    w.gram = (double*)(p + L.off[10]);
    w.pscr = (double*)(p + L.off[11]);
    w.jscr = (double*)(p + L.off[12]);
    w.D = (double*)(p + L.off[13]);
    w.Us = (double*)(p + L.off[14]);
    w.Vs = (double*)(p + L.off[15]);
    w.bars = (unsigned*)(p + L.off[16]);
    w.counters = (int*)(p + L.off[17]);
    w.status = (int*)(p + L.off[18]);
    w.part_elems = L.part_elems;
    return w;
}

// Grow-only workspace cached per device (freed at process exit by the driver).
struct CachedWs {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_ws_mu;
std::unordered_map<int, CachedWs> g_ws;

cudaError_t cached_workspace(int dev, size_t bytes, void** out) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    CachedWs& c = g_ws[dev];
    if (c.bytes < bytes) {
        if (c.ptr) {
            cudaDeviceSynchronize();
            cudaFree(c.ptr);
            c.ptr = nullptr;
            c.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&c.ptr, bytes);
        if (e != cudaSuccess) {
            c.ptr = nullptr;
            return e;
        }
        c.bytes = bytes;
    }
    *out = c.ptr;
    return cudaSuccess;
}

#define CK(x)                                 \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

struct Ctx {
    int64_t m, n, ldt;
    int b, q;
    uint64_t seed;
    double *U, *T, *V;
    Workspace w;
    int sms;
    cudaStream_t st;
};

cudaError_t gemm(Ctx& c, const char* role, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    double flops = 2.0 * (double)M * (double)N * (double)K;
    double bytes = 8.0 * ((double)M * K + (double)K * N + (double)M * N * (beta != 0.0 ? 2.0 : 1.0));
    TraceScope ts(role, flops, bytes, c.st);
    return gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.part, c.w.part_elems, c.sms, c.st);
}

// Householder QR of a len x w panel plus its W (explicit) and Tf.
cudaError_t factor_panel(Ctx& c, double* P, int64_t ld, int64_t len, int w) {
    {
        TraceScope ts("panel_qr", 2.0 * (double)len * w * w, 16.0 * (double)len * w, c.st);
        CK(panel_qr(P, ld, len, w, c.w.tau, c.w.pscr, c.w.bars, c.w.status, c.sms, c.st));
    }
    {
        TraceScope ts("extract_w", 0.0, 16.0 * (double)len * w, c.st);
        CK(extract_w(P, ld, len, w, c.w.W, c.st));
    }
    CK(gemm(c, "gemm_gram", true, false, w, w, len, 1.0, c.w.W, len, c.w.W, len, 0.0, c.w.gram, w));
    TraceScope ts("tfactor", (double)w * w * w / 3.0, 16.0 * (double)w * w, c.st);
    return tfactor(c.w.gram, c.w.tau, w, c.w.Tf, c.w.status, c.st);
}

// C (rows x cols) := C (I - W Tf W^T), W = c.w.W (cols x w), Tf = c.w.Tf.
cudaError_t apply_right(Ctx& c, double* C, int64_t ldc, int64_t rows, int64_t cols, int w) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    CK(gemm(c, "gemm_right", false, false, rows, w, cols, 1.0, C, ldc, c.w.W, cols, 0.0, c.w.X, rows));
    CK(gemm(c, "gemm_right_tf", false, false, rows, w, w, 1.0, c.w.X, rows, c.w.Tf, w, 0.0, c.w.X2, rows));
    return gemm(c, "gemm_right", false, true, rows, cols, w, -1.0, c.w.X2, rows, c.w.W, cols, 1.0, C, ldc);
}

// C (len x cols) := (I - W Tf W^T)^T C, W = c.w.W (len x w).
cudaError_t apply_left_t(Ctx& c, double* C, int64_t ldc, int64_t len, int64_t cols, int w) {
    if (len <= 0 || cols <= 0) return cudaSuccess;
    CK(gemm(c, "gemm_left", true, false, w, cols, len, 1.0, c.w.W, len, C, ldc, 0.0, c.w.X, w));
    CK(gemm(c, "gemm_left_tf", true, false, w, cols, w, 1.0, c.w.Tf, w, c.w.X, w, 0.0, c.w.X2, w));
    return gemm(c, "gemm_left", false, false, len, cols, w, -1.0, c.w.W, len, c.w.X2, w, 1.0, C, ldc);
}

// Panel QR of T(k0:m, k0:k0+w), left update, small SVD and its application.
cudaError_t panel_and_svd(Ctx& c, int64_t k0, int w) {
    const int64_t m = c.m, n = c.n, ldt = c.ldt;
    const int64_t mp = m - k0;
    double* T = c.T;
    double* P = T + k0 + k0 * ldt;
    CK(factor_panel(c, P, ldt, mp, w));
    CK(apply_left_t(c, T + k0 + (k0 + w) * ldt, ldt, mp, n - k0 - w, w));
    if (c.U) CK(apply_right(c, c.U + k0 * m, m, m, mp, w));
    {
        TraceScope tsv("jacobi_svd", 0.0, 8.0 * 3.0 * (double)w * w, c.st);
        CK(jacobi_svd(P, ldt, w, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status,
                      kMaxSweeps, c.st));
    }
    if (k0 > 0) {  // T(0:k0, blk) := T(0:k0, blk) Vs
        CK(gemm(c, "gemm_svdapply", false, false, k0, w, w, 1.0, T + k0 * ldt, ldt, c.w.Vs, w, 0.0, c.w.tmp, k0));
        CK(copy_matrix(c.w.tmp, k0, T + k0 * ldt, ldt, k0, w, c.st));
    }
    int64_t nr = n - k0 - w;
    if (nr > 0) {  // T(blk, k0+w:n) := Us^T T(blk, k0+w:n)
        CK(gemm(c, "gemm_svdapply", true, false, w, nr, w, 1.0, c.w.Us, w, T + k0 + (k0 + w) * ldt, ldt, 0.0, c.w.tmp, w));
        CK(copy_matrix(c.w.tmp, w, T + k0 + (k0 + w) * ldt, ldt, w, nr, c.st));
    }
    CK(set_diag_block(T, ldt, k0, m, w, c.w.D, c.st));
    if (c.V) {
        CK(gemm(c, "gemm_svdapply", false, false, n, w, w, 1.0, c.V + k0 * n, n, c.w.Vs, w, 0.0, c.w.tmp, n));
        CK(copy_matrix(c.w.tmp, n, c.V + k0 * n, n, n, w, c.st));
    }
    if (c.U) {
        CK(gemm(c, "gemm_svdapply", false, false, m, w, w, 1.0, c.U + k0 * m, m, c.w.Us, w, 0.0, c.w.tmp, m));
        CK(copy_matrix(c.w.tmp, m, c.U + k0 * m, m, m, w, c.st));
    }
    return cudaSuccess;
}

// One sketch step (n' > b) at column offset k0.
cudaError_t sketch_step(Ctx& c, int64_t i) {
    const int64_t m = c.m, n = c.n, ldt = c.ldt;
    const int b = c.b;
    const int64_t k0 = i * (int64_t)b, mp = m - k0, np = n - k0;
    double* T22 = c.T + k0 + k0 * ldt;
    {
        TraceScope ts("gaussian", 0.0, 8.0 * (double)mp * b, c.st);
        CK(gaussian_f64(c.seed, i, mp, b, c.w.G, mp, c.st));
    }
    CK(gemm(c, "gemm_sketch", true, false, np, b, mp, 1.0, T22, ldt, c.w.G, mp, 0.0, c.w.Y, np));
    for (int it = 0; it < c.q; ++it) {
        CK(gemm(c, "gemm_sketch", false, false, mp, b, np, 1.0, T22, ldt, c.w.Y, np, 0.0, c.w.Z, mp));
        CK(gemm(c, "gemm_sketch", true, false, np, b, mp, 1.0, T22, ldt, c.w.Z, mp, 0.0, c.w.Y, np));
    }
    CK(factor_panel(c, c.w.Y, np, np, b));
    CK(apply_right(c, c.T + k0 * ldt, ldt, m, np, b));
    if (c.V) CK(apply_right(c, c.V + k0 * n, n, n, np, b));
    return panel_and_svd(c, k0, b);
}

cudaError_t run_factor(Ctx& c, const double* A, int64_t lda, int64_t stop_after) {
    const int64_t m = c.m, n = c.n;
    if (A != c.T) CK(copy_matrix(A, lda, c.T, c.ldt, m, n, c.st));
    if (c.U) CK(set_identity(c.U, m, m, c.st));
    if (c.V) CK(set_identity(c.V, n, n, c.st));
    CK(check_finite(c.T, c.ldt, m, n, c.w.status, c.st));
    for (int64_t i = 0;; ++i) {
        if (stop_after >= 0 && i >= stop_after) break;
        int64_t k0 = i * (int64_t)c.b;
        int64_t np = n - k0;
        if (np <= 0) break;
        if (np <= c.b) {
            CK(panel_and_svd(c, k0, (int)np));
            break;
        }
        CK(sketch_step(c, i));
    }
    return cudaSuccess;
}

randutv_status status_from_bits(int bits) {
    if (bits & ST_NONFINITE) return RANDUTV_ENONFINITE;
    if (bits & ST_TIMEOUT) return RANDUTV_ETIMEOUT;
    if (bits & ST_NOCONV) return RANDUTV_ENOCONV;
    return RANDUTV_OK;
}

bool args_ok(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, const double* T) {
    if (m < 0 || n < 0 || m < n || b < 1 || q < 0) return false;
    if (lda < std::max<int64_t>(m, 1)) return false;
    if (n > 0 && (A == nullptr || T == nullptr)) return false;
    if (m > (int64_t)1 << 30 || b > 512) return false;
    return true;
}

}  // namespace

}  // namespace rutv

using namespace rutv;

extern "C" {

const char* randutv_status_string(int s) {
    switch (s) {
        case RANDUTV_OK: return "ok";
        case RANDUTV_EINVAL: return "invalid argument";
        case RANDUTV_ENOMEM: return "out of device memory";
        case RANDUTV_ENONFINITE: return "non-finite value met";
        case RANDUTV_ENOCONV: return "Jacobi SVD hit its sweep cap";
        case RANDUTV_ETIMEOUT: return "bounded device wait timed out";
        case RANDUTV_ECUDA: return "CUDA runtime error";
        case RANDUTV_ENOTIMPL: return "not implemented";
        default: return "unknown status";
    }
}

size_t randutv_workspace_size(int64_t m, int64_t n, int b, int prec) {
    if (m < n || n < 0 || b < 1) return 0;
    if (prec != RANDUTV_FP64) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return make_layout(m, n, b, device_sms(dev)).total;
}

randutv_status randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed,
                                 double* U, double* T, double* V, int prec, void* stream, void* workspace,
                                 size_t ws_bytes, int64_t stop_after, int* info) {
    if (!args_ok(m, n, A, lda, b, q, T)) return RANDUTV_EINVAL;
    if (prec != RANDUTV_FP64) return RANDUTV_ENOTIMPL;
    if (A == T && lda != m) return RANDUTV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RANDUTV_ECUDA;
    const int sms = device_sms(dev);
    Layout L = make_layout(m, n, b, sms);
    void* base = workspace;
    if (base == nullptr) {
        if (cached_workspace(dev, L.total, &base) != cudaSuccess) return RANDUTV_ENOMEM;
    } else if (ws_bytes < L.total) {
        return RANDUTV_ENOMEM;
    }
    Ctx c{};
    c.m = m; c.n = n; c.ldt = std::max<int64_t>(m, 1);
    c.b = b; c.q = q; c.seed = seed;
    c.U = U; c.T = T; c.V = V;
    c.w = carve(base, L);
    c.sms = sms;
    c.st = st;
    if (cudaMemsetAsync(c.w.status, 0, sizeof(int), st) != cudaSuccess) return RANDUTV_ECUDA;
    if (m == 0) return RANDUTV_OK;
    if (run_factor(c, A, lda, stop_after) != cudaSuccess) return RANDUTV_ECUDA;
    if (info != nullptr) {
        if (cudaMemcpyAsync(info, c.w.status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RANDUTV_ECUDA;
        return RANDUTV_OK;
    }
    int bits = 0;
    if (cudaMemcpyAsync(&bits, c.w.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return RANDUTV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RANDUTV_ECUDA;
    return status_from_bits(bits);
}

randutv_status randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed,
                              double* U, double* T, double* V) {
    return randutv_factor_ex(m, n, A, lda, b, q, seed, U, T, V, RANDUTV_FP64, nullptr, nullptr, 0, -1, nullptr);
}

randutv_status randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                   uint64_t seed, double* U, double* T, double* V, int prec) {
    if (!args_ok(m, n, A, lda, b, q, T)) return RANDUTV_EINVAL;
    double *dA = nullptr, *dU = nullptr, *dV = nullptr;
    size_t bytesT = sizeof(double) * (size_t)m * n;
    randutv_status rs = RANDUTV_OK;
    if (cudaMalloc(&dA, std::max<size_t>(bytesT, 8)) != cudaSuccess) return RANDUTV_ENOMEM;
    if (U && cudaMalloc(&dU, std::max<size_t>(sizeof(double) * (size_t)m * m, 8)) != cudaSuccess) rs = RANDUTV_ENOMEM;
    if (rs == RANDUTV_OK && V && cudaMalloc(&dV, std::max<size_t>(sizeof(double) * (size_t)n * n, 8)) != cudaSuccess)
        rs = RANDUTV_ENOMEM;
    if (rs == RANDUTV_OK && bytesT > 0 &&
        cudaMemcpy2D(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m, n,
                     cudaMemcpyHostToDevice) != cudaSuccess)
        rs = RANDUTV_ECUDA;
    if (rs == RANDUTV_OK)
        rs = randutv_factor_ex(m, n, dA, m, b, q, seed, U ? dU : nullptr, dA, V ? dV : nullptr, prec, nullptr,
                               nullptr, 0, -1, nullptr);
    if ((rs == RANDUTV_OK || rs == RANDUTV_ENOCONV) && bytesT > 0) {
        if (cudaMemcpy(T, dA, bytesT, cudaMemcpyDeviceToHost) != cudaSuccess) rs = RANDUTV_ECUDA;
        if (U && cudaMemcpy(U, dU, sizeof(double) * (size_t)m * m, cudaMemcpyDeviceToHost) != cudaSuccess)
            rs = RANDUTV_ECUDA;
        if (V && cudaMemcpy(V, dV, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost) != cudaSuccess)
            rs = RANDUTV_ECUDA;
    }
    cudaFree(dA);
    if (dU) cudaFree(dU);
    if (dV) cudaFree(dV);
    return rs;
}

}  // extern "C"
