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
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/randutv.h"
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace rutv {

namespace {
std::atomic<long long> g_wait_limit{kSpinLimit};
std::atomic<int> g_sweep_cap{30};
}  // namespace

namespace {
thread_local DevGate t_gate{nullptr, 0};
}  // namespace

const DevGate& current_gate() { return t_gate; }
GateScope::GateScope(const int* flag, int need) : saved_flag_(t_gate.flag), saved_need_(t_gate.need) {
    t_gate = DevGate{flag, need};
}
GateScope::~GateScope() { t_gate = DevGate{saved_flag_, saved_need_}; }

long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }
int sweep_cap() { return g_sweep_cap.load(std::memory_order_relaxed); }

namespace {

constexpr size_t kAlign = 256;
constexpr int kDefaultSweeps = 30;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Workspace {
    double *G, *Y, *Z, *W, *X, *X2, *tmp, *part, *tau, *Tf, *gram, *pscr, *jscr, *D, *Us, *Vs;
    unsigned* bars;
    int* counters;
    int* status;
    size_t part_elems;
    // low-precision sketch (null for RANDUTV_FP64)
    uint16_t *S, *St, *B16;
    float *Pf, *Xf, *cqr;
    unsigned long long* amax;
    // learned q
    float* feat;      // 16 features of the current block
    int* qdev;        // chosen q
    double* dq;       // candidate diagonals, 4 x w (trace mode)
    double* rdiag;    // learned q / trace: the R diagonal of the last panel QR (w)
    double* sdiag;    // learned q / trace: |R_jj| of the compressed sketch (w)
    double* level;    // learned q / trace: the compressed sketch's norm, and the first block's (2)
    double* W2;       // left update from the old split: W_V(b:, :) ((n' - b) x b), or null
    float* qmodel;    // network parameters on the device
    void* oz;         // digit slices and exponents of the emulated FP64 products
    size_t oz_bytes;
    void* oz_rows;    // digit planes of T(:, k0:n) split by rows (kept for one step)
    void* oz_cols;    // digit planes of T22 split by columns (kept for one step)
    size_t oz_rows_bytes;  // size of oz_rows (reused by the grouped U / V accumulation)
    double* svdp;     // FP32-preconditioned SVD: Q, Q', Gram, triu(R), R Q (w x w each), or null
    double* defer;    // reflectors and small factors kept for the deferred U / V accumulation
    size_t defer_elems;
    // the side stream's own scratch (the small SVD and its application run there)
    void* oz2;
    size_t oz2_bytes;
    double* tmp2;
    double* part2;
    int* qlog;        // learned mode: the q chosen at each sketch step (-1: none)
};

constexpr int kSlots = 38;
struct Layout {
    size_t off[kSlots];
    size_t total;
    size_t part_elems;
    int64_t wmax;  // the widest block: min(b, n)
};

int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

// widths whose b x b SVD takes the FP32-preconditioned route
bool svd_precond_width(int w) { return w >= 64 && w <= 128; }

// Doubles kept for the deferred accumulation of U and V: per block step the
// reflectors W_V ((n - k0) x b) and W_U ((m - k0) x w), T_V, T_U, V_s, U_s
// (w x w each).
size_t defer_elems(int64_t m, int64_t n, int b) {
    size_t e = 0;
    for (int64_t k0 = 0; k0 < n; k0 += b) {
        const int64_t w = std::min<int64_t>(b, n - k0);
        e += (size_t)(n - k0) * b + (size_t)(m - k0) * w + 4 * (size_t)b * b;
    }
    return e;
}

// Doubles kept by the QR-first phase: per panel of b columns its W
// ((m - k0) x w) and its triangular factor (w x w).
size_t qr_defer_elems(int64_t m, int64_t n, int b) {
    size_t e = 0;
    for (int64_t k0 = 0; k0 < n; k0 += b) {
        const int64_t w = std::min<int64_t>(b, n - k0);
        e += (size_t)(m - k0) * w + (size_t)w * w;
    }
    return e;
}

bool lowp_prec(int prec) {
    return prec == RANDUTV_SKETCH_BF16 || prec == RANDUTV_SKETCH_FP16_SCALED || prec == RANDUTV_EMULATED_SKETCH_BF16;
}
bool emulated_prec(int prec) { return prec == RANDUTV_FP64_EMULATED || prec == RANDUTV_EMULATED_SKETCH_BF16; }
bool valid_prec(int prec) { return prec == RANDUTV_FP64 || lowp_prec(prec) || emulated_prec(prec); }

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

Layout make_layout(int64_t m, int64_t n, int b, int sms, int prec, bool qr_first = false) {
    Layout L{};
    int64_t mx = std::max<int64_t>(std::max(m, n), 1);
    int64_t bb = std::max(b, 1);
    int64_t wmax = std::min<int64_t>(bb, std::max<int64_t>(n, 1));
    size_t part = (size_t)8 * sms * 64 * 64 + (size_t)2 * mx * wmax;
    const bool lp = lowp_prec(prec);
    const int64_t npad = lp ? tc_gemm_npad((int)wmax) : 0;
    size_t sizes[kSlots] = {
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
        lp ? sizeof(uint16_t) * (size_t)n * round8(m) : 0,          // S  = T22 col-major, 16-bit
        lp ? sizeof(uint16_t) * (size_t)m * round8(n) : 0,          // St = T22 row-major, 16-bit
        lp ? sizeof(uint16_t) * (size_t)npad * round8(mx) : 0,      // 16-bit B operand (G, Y, Z)
        lp ? sizeof(float) * (size_t)8 * mx * npad : 0,             // split-K partials (FP32)
        lp ? sizeof(float) * (size_t)mx * npad : 0,                 // Y / Z in FP32
        lp ? sizeof(float) * cholqr_scratch_floats((int)npad, sms) : 0,
        lp ? sizeof(unsigned long long) : 0,                        // max |T22|
        sizeof(float) * 32 + sizeof(double) * (6 * (size_t)wmax + 2),  // learned-q features, q, candidates, R diagonals
        sizeof(float) * (size_t)learnq_nparam(),                    // learned-q model
        emulated_prec(prec) ? oz_work_bytes(mx, std::max<int64_t>(wmax, 128), mx) : 0,   // Ozaki digits
        emulated_prec(prec) ? oz_operand_bytes(m, n) : 0,                               // T(:, k0:n) by rows
        emulated_prec(prec) ? oz_operand_bytes(n, m) : 0,                               // T22 by columns
        svd_precond_width((int)wmax) ? sizeof(double) * 5 * (size_t)wmax * wmax : 0,   // preconditioned SVD
        sizeof(double) * (qr_first ? qr_defer_elems(m, n, b) + defer_elems(n, n, b)
                                   : defer_elems(m, n, b)),                             // deferred U / V
        emulated_prec(prec) ? 2 * oz_operand_bytes(mx, std::max<int64_t>(wmax, 128)) + 8192 : 0,  // side Ozaki
        sizeof(double) * (size_t)mx * wmax,                                             // side tmp
        sizeof(double) * part,                                                          // side partials
        sizeof(int) * (size_t)(n / std::max(b, 1) + 2),                                  // learned q per step
        emulated_prec(prec) ? sizeof(double) * (size_t)mx * wmax : 0};                  // W_V(b:, :)
    size_t o = 0;
    for (int i = 0; i < kSlots; ++i) {
        L.off[i] = o;
        o += align_up(sizes[i]);
    }
    L.total = o;
    L.part_elems = part;
    L.wmax = wmax;
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
    w.S = (uint16_t*)(p + L.off[19]);
    w.St = (uint16_t*)(p + L.off[20]);
    w.B16 = (uint16_t*)(p + L.off[21]);
    w.Pf = (float*)(p + L.off[22]);
    w.Xf = (float*)(p + L.off[23]);
    w.cqr = (float*)(p + L.off[24]);
    w.amax = (unsigned long long*)(p + L.off[25]);
    w.feat = (float*)(p + L.off[26]);
    w.qdev = (int*)(w.feat + 16);
    w.dq = (double*)(p + L.off[26] + sizeof(float) * 32);
    w.rdiag = w.dq + 4 * (size_t)L.wmax;
    w.sdiag = w.rdiag + (size_t)L.wmax;
    w.level = w.sdiag + (size_t)L.wmax;
    w.qmodel = (float*)(p + L.off[27]);
    w.oz = (void*)(p + L.off[28]);
    w.oz_bytes = L.off[29] - L.off[28];
    w.oz_rows = L.off[30] > L.off[29] ? (void*)(p + L.off[29]) : nullptr;
    w.oz_cols = L.off[31] > L.off[30] ? (void*)(p + L.off[30]) : nullptr;
    w.oz_rows_bytes = L.off[30] - L.off[29];
    w.svdp = L.off[32] > L.off[31] ? (double*)(p + L.off[31]) : nullptr;
    w.defer = (double*)(p + L.off[32]);
    w.defer_elems = (L.off[33] - L.off[32]) / sizeof(double);
    w.oz2 = (void*)(p + L.off[33]);
    w.oz2_bytes = L.off[34] - L.off[33];
    w.tmp2 = (double*)(p + L.off[34]);
    w.part2 = (double*)(p + L.off[35]);
    w.qlog = (int*)(p + L.off[36]);
    w.W2 = L.total > L.off[37] ? (double*)(p + L.off[37]) : nullptr;
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

// Grow-only device buffers for the host-buffer entry point (A/T, U, V),
// cached per device like the workspace.
std::mutex g_buf_mu;
std::unordered_map<int, CachedWs> g_buf[3];

cudaError_t cached_buffer(int dev, int slot, size_t bytes, void** out) {
    std::lock_guard<std::mutex> lk(g_buf_mu);
    CachedWs& c = g_buf[slot][dev];
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

// A second stream and two events per device: the FP32 Jacobi of a block step
// runs on it while the left update of the same step runs on the caller's
// stream.  Created on first use, kept for the life of the process.
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;      // FP32 Jacobi overlapping the left update
    cudaEvent_t panel = nullptr, right = nullptr;     // main -> side: panel factored, right update done
    cudaEvent_t applied = nullptr;                    // side -> main: small SVD applied to T
    cudaEvent_t svd_done = nullptr;                   // side -> main: small SVD computed (D ready)
    cudaEvent_t merged[2] = {nullptr, nullptr};       // side -> main: a U/V group's WY form merged
    cudaEvent_t freed[2] = {nullptr, nullptr};        // main -> side: that merge buffer applied
};
std::mutex g_side_mu;
std::unordered_map<int, SideStream> g_side;

cudaError_t side_stream(SideStream** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_side_mu);
    SideStream& s = g_side[dev];
    if (!s.st) {
        if ((e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.ready, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.panel, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.right, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.applied, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&s.svd_done, cudaEventDisableTiming)) != cudaSuccess) return e;
        for (int k = 0; k < 2; ++k) {
            if ((e = cudaEventCreateWithFlags(&s.merged[k], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&s.freed[k], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
    }
    *out = &s;
    return cudaSuccess;
}

// Calls on one device share its side stream and events, so their launch
// sequences must not interleave: each call enqueues its whole factorization
// under its device's lock.  The GPU work of calls on different streams still
// overlaps.
std::mutex g_enqueue_mu[64];
std::mutex& enqueue_lock(int dev) { return g_enqueue_mu[(unsigned)dev % 64u]; }

enum SketchMode { MODE_FIXED = 0, MODE_LEARNED = 1, MODE_TRACE = 2 };

// Splits of the trailing matrix reused by the emulated products of one block
// step while T is unchanged: T(:, k0:n) by rows serves Z = T22 Y (rows k0:m)
// and the right update's T(:, k0:n) W_V; T22 by columns serves Y = T22^T Z.
struct OzCache {
    int64_t k0 = -1;
    bool rows = false, cols = false;
    OzOperand r{}, c{};
};

struct Ctx {
    int64_t m, n, ldt;
    int b, q, prec;
    int mode = MODE_FIXED;
    bool have_model = false;
    float* tr_feat = nullptr;         // host, 16 per block (trace mode)
    int* tr_label = nullptr;          // host, one per block (trace mode)
    double* tr_cand = nullptr;        // host, 4 x b per block (trace mode), optional
    int64_t tr_max = 0, tr_count = 0;
    int64_t tr_stride = 1;            // trace mode: record every tr_stride-th sketch step ...
    int64_t tr_offset = 0;            // ... starting at this one
    uint64_t seed;
    double *U, *T, *V;
    Workspace w;
    OzCache oc;
    // left update of the current sketch step from the column split of T22
    // made before the right update (left_from_old_split_prepare)
    bool left_old = false;
    OzOperand left_cols{};
    int sms;
    cudaStream_t st;
    // deferred U / V: what each block step left in w.defer
    struct Step {
        int64_t k0;
        int w;
        bool sketch;
        size_t wv, tv, wu, tu, us, vs;  // offsets into w.defer (wv, tv unused without a sketch)
    };
    std::vector<Step> steps;
    size_t defer_top = 0;
    // QR-first phase (Sec. 5.1): each panel's W and triangular factor
    struct QrStep {
        int64_t k0;
        int w;
        size_t wu, tu;
    };
    std::vector<QrStep> qr;
    int64_t ldu = 0, ldv = 0;      // leading dimensions of U and V
    // tolerance stop and resume
    double rank_tol = 0.0, t00 = 0.0;
    int64_t cols_done = 0, rank = 0;
    int64_t start_step = 0;
    bool resume = false;
    std::vector<double> dhost;     // the last block's diagonal, read by the host
    // overlap of the small SVD with the next block step (fixed-q mode)
    bool overlap = false;
    int64_t pending = -1;        // step whose small SVD still has to be applied to T
    bool applied_pending = false;  // an application was queued that the main stream has not waited for
};

cudaError_t gemm(Ctx& c, const char* role, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    double flops = 2.0 * (double)M * (double)N * (double)K;
    double bytes = 8.0 * ((double)M * K + (double)K * N + (double)M * N * (beta != 0.0 ? 2.0 : 1.0));
    TraceScope ts(role, flops, bytes, c.st);
    if (emulated_prec(c.prec) && M >= 128 && N >= 64 && K >= 64)
        return oz_gemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.oz, c.w.oz_bytes, c.sms, c.w.status,
                       c.st);
    return gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.part, c.w.part_elems, c.sms, c.st);
}

bool oz_shape(const Ctx& c, int64_t M, int64_t N, int64_t K) {
    return emulated_prec(c.prec) && c.w.oz_rows != nullptr && M >= 128 && N >= 64 && K >= 64;
}

const OzOperand* oz_rows_of(Ctx& c, int64_t k0, cudaError_t* e) {
    if (c.oc.k0 != k0) c.oc = OzCache{k0};
    if (!c.oc.rows) {
        TraceScope ts("oz_split_cached", 0.0, 24.0 * (double)c.m * (c.n - k0), c.st);
        *e = oz_split(false, c.T + k0 * c.ldt, c.ldt, c.m, c.n - k0, c.w.oz_rows, &c.oc.r, c.w.status, c.st);
        c.oc.rows = (*e == cudaSuccess);
    }
    return &c.oc.r;
}

const OzOperand* oz_cols_of(Ctx& c, int64_t k0, cudaError_t* e) {
    if (c.oc.k0 != k0) c.oc = OzCache{k0};
    if (!c.oc.cols) {
        TraceScope ts("oz_split_cached", 0.0, 24.0 * (double)(c.m - k0) * (c.n - k0), c.st);
        *e = oz_split(true, c.T + k0 + k0 * c.ldt, c.ldt, c.n - k0, c.m - k0, c.w.oz_cols, &c.oc.c, c.w.status,
                      c.st);
        c.oc.cols = (*e == cudaSuccess);
    }
    return &c.oc.c;
}

// Y (M x w) = La(a0 : a0 + M, :) B with La a cached split and B (K x w,
// column-major) split afresh.
cudaError_t oz_cached_product(Ctx& c, const char* role, const OzOperand& a, int64_t a0, int64_t M, int w,
                              const double* B, int64_t ldb, double* Y, int64_t ldy) {
    const int64_t K = a.K;
    TraceScope ts(role, 2.0 * (double)M * w * K, 8.0 * ((double)M * K + (double)K * w + (double)M * w), c.st);
    char* p = (char*)c.w.oz;
    OzOperand bo;
    CK(oz_split(true, B, ldb, w, K, p, &bo, c.w.status, c.st));
    p += oz_operand_bytes(w, K);
    double* P = (double*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    const size_t used = (size_t)((char*)P - (char*)c.w.oz);
    return oz_product(a, a0, bo, 0, M, w, 1.0, 0.0, Y, ldy, P, c.w.oz_bytes > used ? c.w.oz_bytes - used : 0, c.sms,
                      c.w.status, c.st);
}

// Sketch product with the trailing matrix T22 = T(k0:m, k0:n):
// Y = T22^T B (tr) or Y = T22 B; B is K x b.
cudaError_t sketch_gemm(Ctx& c, bool tr, int64_t k0, const double* B, int64_t ldb, double* Y, int64_t ldy) {
    const int64_t mp = c.m - k0, np = c.n - k0;
    const int64_t M = tr ? np : mp, K = tr ? mp : np;
    if (!oz_shape(c, M, c.b, K))
        return gemm(c, "gemm_sketch", tr, false, M, c.b, K, 1.0, c.T + k0 + k0 * c.ldt, c.ldt, B, ldb, 0.0, Y, ldy);
    cudaError_t e = cudaSuccess;
    const OzOperand* a = tr ? oz_cols_of(c, k0, &e) : oz_rows_of(c, k0, &e);
    CK(e);
    return oz_cached_product(c, "gemm_sketch", *a, tr ? 0 : k0, M, c.b, B, ldb, Y, ldy);
}

// Copies a rows x cols matrix (ld lds) into the deferred store; returns its offset.
cudaError_t defer_put(Ctx& c, const double* src, int64_t lds, int64_t rows, int64_t cols, size_t* off,
                      cudaStream_t st) {
    *off = c.defer_top;
    const size_t need = (size_t)rows * cols;
    if (c.defer_top + need > c.w.defer_elems) return cudaErrorInvalidValue;
    c.defer_top += need;
    return copy_matrix(src, lds, c.w.defer + *off, rows, rows, cols, st);
}
cudaError_t defer_put(Ctx& c, const double* src, int64_t lds, int64_t rows, int64_t cols, size_t* off) {
    return defer_put(c, src, lds, rows, cols, off, c.st);
}

// SMs for the cooperative panel QR: with the small SVD overlapping on the
// side stream, room is left for its 16-block cluster and the FP32 block.
int panel_sms(const Ctx& c) { return (c.overlap && c.sms > 64) ? c.sms - 17 : c.sms; }

// Sub-panel width of the blocked panel QR (emulated products only).
constexpr int kSubPanel = 32;

// A product of the blocked panel: emulated on the tensor cores when the
// emulated precision is selected (skinny shapes allowed), else FP64 DMMA.
cudaError_t panel_gemm(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    if (emulated_prec(c.prec) && M >= 16 && N >= 8 && K >= 8)
        return oz_gemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.oz, c.w.oz_bytes, c.sms, c.w.status,
                       c.st);
    return gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.part, c.w.part_elems, c.sms, c.st);
}

// Blocked Householder QR of a len x w panel (the recursion-free form of
// LAPACK's blocked QR, Sec. 2.3): sub-panels of kSubPanel columns are factored
// by the one-barrier-per-column kernel, which also returns each one's compact
// WY form (W_k, Tf_k), and Q_k = I - W_k Tf_k W_k^T is applied to the columns
// right of it, C := Q_k^T C = C - W_k Tf_k^T (W_k^T C), by three products.
// Most of the panel's FP64 multiply-adds thus move into those products
// (emulated on the tensor cores); the reflectors, tau and R are those of the
// unblocked factorization, up to rounding.  Uses c.w.W and c.w.Tf as scratch
// (factor_panel recomputes W, Tf of the whole panel afterwards) and keeps the
// two wk x rest products in c.w.gram: 2 wk (w - wk) <= w^2 for every w.
cudaError_t blocked_panel_qr(Ctx& c, double* P, int64_t ld, int64_t len, int w) {
    for (int k0 = 0; k0 < w; k0 += kSubPanel) {
        const int wk = std::min(kSubPanel, w - k0);
        const int64_t lk = len - k0;
        const int rest = w - k0 - wk;
        double* Pk = P + k0 + (int64_t)k0 * ld;
        if (rest <= 0 || lk <= 0) {
            TraceScope ts("panel_qr", 2.0 * (double)lk * wk * wk, 16.0 * (double)lk * wk, c.st);
            CK(panel_qr(Pk, ld, lk, wk, c.w.tau + k0, c.w.pscr, c.w.bars, c.w.status, panel_sms(c), c.st));
            continue;
        }
        {
            TraceScope ts("panel_qr", 3.0 * (double)lk * wk * wk, 24.0 * (double)lk * wk, c.st);
            CK(panel_qr_wy(Pk, ld, lk, wk, c.w.tau + k0, c.w.W, c.w.Tf, c.w.pscr, c.w.bars, c.w.status,
                           panel_sms(c), c.st));
        }
        TraceScope ts("panel_update", 4.0 * (double)lk * wk * rest, 8.0 * (double)lk * (wk + 2 * rest), c.st);
        double* C = Pk + (int64_t)wk * ld;
        double* Xk = c.w.gram;
        double* X2k = Xk + (size_t)wk * rest;
        CK(panel_gemm(c, true, false, wk, rest, lk, 1.0, c.w.W, lk, C, ld, 0.0, Xk, wk));
        CK(gemm_f64(true, false, wk, rest, wk, 1.0, c.w.Tf, wk, Xk, wk, 0.0, X2k, wk, c.w.part, c.w.part_elems, c.sms,
                    c.st));
        CK(panel_gemm(c, false, false, lk, rest, wk, -1.0, c.w.W, lk, X2k, wk, 1.0, C, ld));
    }
    return cudaSuccess;
}

// Householder QR of a len x w panel plus its W (explicit) and Tf.
cudaError_t factor_panel(Ctx& c, double* P, int64_t ld, int64_t len, int w) {
    if (emulated_prec(c.prec) && w > kSubPanel && len >= 1024) {
        CK(blocked_panel_qr(c, P, ld, len, w));
    } else {
        TraceScope ts("panel_qr", 2.0 * (double)len * w * w, 16.0 * (double)len * w, c.st);
        CK(panel_qr(P, ld, len, w, c.w.tau, c.w.pscr, c.w.bars, c.w.status, panel_sms(c), c.st));
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

// T(:, k0:n) := T(:, k0:n) (I - W Tf W^T) with the first product taken from
// the cached row split of T(:, k0:n); T changes, so the cache is dropped.
cudaError_t apply_right_T(Ctx& c, int64_t k0, int w) {
    const int64_t rows = c.m, cols = c.n - k0;
    double* C = c.T + k0 * c.ldt;
    if (!oz_shape(c, rows, w, cols)) {
        c.oc = OzCache{};
        return apply_right(c, C, c.ldt, rows, cols, w);
    }
    cudaError_t e = cudaSuccess;
    const OzOperand* a = oz_rows_of(c, k0, &e);
    CK(e);
    CK(oz_cached_product(c, "gemm_right", *a, 0, rows, w, c.w.W, cols, c.w.X, rows));
    c.oc = OzCache{};
    CK(gemm(c, "gemm_right_tf", false, false, rows, w, w, 1.0, c.w.X, rows, c.w.Tf, w, 0.0, c.w.X2, rows));
    return gemm(c, "gemm_right", false, true, rows, cols, w, -1.0, c.w.X2, rows, c.w.W, cols, 1.0, C, c.ldt);
}

// C (len x cols) := (I - W Tf W^T)^T C, W = c.w.W (len x w).
cudaError_t apply_left_t(Ctx& c, double* C, int64_t ldc, int64_t len, int64_t cols, int w) {
    if (len <= 0 || cols <= 0) return cudaSuccess;
    CK(gemm(c, "gemm_left", true, false, w, cols, len, 1.0, c.w.W, len, C, ldc, 0.0, c.w.X, w));
    CK(gemm(c, "gemm_left_tf", true, false, w, cols, w, 1.0, c.w.Tf, w, c.w.X, w, 0.0, c.w.X2, w));
    return gemm(c, "gemm_left", false, false, len, cols, w, -1.0, c.w.W, len, c.w.X2, w, 1.0, C, ldc);
}

// SVD of the w x w upper triangle of R (Sec. 3.2.3).  For 64 <= w <= 128 the
// FP64 Jacobi is preconditioned: an FP32 Jacobi gives Q (orthogonal to about
// 1e-6), two Newton-Schulz steps Q := Q (3I - Q^T Q) / 2 make it orthogonal
// to FP64 rounding, and the FP64 Jacobi then runs on R Q with V starting at
// Q, so Vs = Q W and R = Us diag(D) Vs^T as before, after a few sweeps.
// First half: the FP32 Jacobi (w x w, one block) on a side stream, started
// right after the panel QR so that it overlaps the left update; R (the
// upper triangle of the panel's first w columns) is not touched by that
// update.  Returns whether the preconditioned route was started.
cudaError_t svd_block_begin(Ctx& c, const double* R, int64_t ldr, int w, bool* started) {
    *started = false;
    if (!c.w.svdp || !svd_precond_width(w)) return cudaSuccess;
    SideStream* ss = nullptr;
    CK(side_stream(&ss));
    CK(cudaEventRecord(ss->ready, c.st));
    CK(cudaStreamWaitEvent(ss->st, ss->ready, 0));
    {
        TraceScope t32("jacobi_fp32", 0.0, 0.0, ss->st);
        CK(jacobi32_precondition(R, ldr, w, c.w.svdp, 8, ss->st));
    }
    CK(cudaEventRecord(ss->done, ss->st));
    *started = true;
    return cudaSuccess;
}

// SVD of the w x w upper triangle of R (Sec. 3.2.3).  For 64 <= w <= 128 the
// FP64 Jacobi is preconditioned: an FP32 Jacobi gives Q (orthogonal to about
// 1e-6; started by svd_block_begin), two Newton-Schulz steps
// Q := Q (3I - Q^T Q) / 2 make it orthogonal to FP64 rounding, and the FP64
// Jacobi then runs on R Q with V starting at Q, so Vs = Q W and
// R = Us diag(D) Vs^T as before, after a few sweeps.
cudaError_t svd_block(Ctx& c, const double* R, int64_t ldr, int w, bool started) {
    TraceScope tsv("jacobi_svd", 0.0, 8.0 * 3.0 * (double)w * w, c.st);
    if (!started)
        return jacobi_svd(R, ldr, w, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status,
                          sweep_cap(), c.st);
    SideStream* ss = nullptr;
    CK(side_stream(&ss));
    CK(cudaStreamWaitEvent(c.st, ss->done, 0));
    const size_t w2 = (size_t)w * w;
    double* Q = c.w.svdp;
    double* Q1 = Q + w2;
    double* G = Q1 + w2;
    double* Ru = G + w2;
    double* X = Ru + w2;
    for (int it = 0; it < 2; ++it) {
        CK(gemm(c, "svd_precond", true, false, w, w, w, 1.0, Q, w, Q, w, 0.0, G, w));
        CK(copy_matrix(Q, w, Q1, w, w, w, c.st));
        CK(gemm(c, "svd_precond", false, false, w, w, w, -0.5, Q, w, G, w, 1.5, Q1, w));
        std::swap(Q, Q1);
    }
    CK(triu_copy(R, ldr, w, Ru, c.st));
    CK(gemm(c, "svd_precond", false, false, w, w, w, 1.0, Ru, w, Q, w, 0.0, X, w));
    TraceScope t64("jacobi_fp64", 0.0, 0.0, c.st);
    return jacobi_svd(X, w, w, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status, sweep_cap(),
                      c.st, true, true, Q);
}

// ---- overlap of the small SVD with the next block step (fixed-q mode) ------
// Step i's b x b SVD needs only its panel QR, and its application to T
// touches columns blk_i and rows blk_i; step i+1's sketch, panel and left
// update touch neither.  So the SVD runs on the side stream while the main
// stream goes on: the side stream waits for the panel, computes the SVD,
// then waits for step i+1's right update and applies Us, Vs.  The rows
// blk_i of T(:, J2') that step i+1's right update reads are then not yet
// multiplied by Us^T; left and right multiplications commute, so applying
// Us^T after that update gives the same T.  The main stream waits for an
// application before the next sketch (the row split of T(:, J2') must see
// it) and before U, V are accumulated.

// A copy of the context that runs on the side stream with its own scratch.
Ctx side_ctx(const Ctx& c, cudaStream_t st2) {
    Ctx c2 = c;
    c2.st = st2;
    c2.w.oz = c.w.oz2;
    c2.w.oz_bytes = c.w.oz2_bytes;
    c2.w.tmp = c.w.tmp2;
    c2.w.part = c.w.part2;
    c2.steps.clear();
    return c2;
}

// The SVD of R (w x w upper triangle) on the side stream, after the panel.
cudaError_t svd_side(Ctx& c, const double* R, int64_t ldr, int w) {
    SideStream* ss = nullptr;
    CK(side_stream(&ss));
    CK(cudaEventRecord(ss->panel, c.st));
    CK(cudaStreamWaitEvent(ss->st, ss->panel, 0));
    Ctx c2 = side_ctx(c, ss->st);
    TraceScope tsv("jacobi_svd", 0.0, 8.0 * 3.0 * (double)w * w, c2.st);
    if (!c.w.svdp || !svd_precond_width(w)) {
        CK(jacobi_svd(R, ldr, w, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status,
                      sweep_cap(), c2.st));
        return cudaEventRecord(ss->svd_done, c2.st);
    }
    const size_t w2 = (size_t)w * w;
    double* Q = c.w.svdp;
    double* Q1 = Q + w2;
    double* G = Q1 + w2;
    double* Ru = G + w2;
    double* X = Ru + w2;
    {
        TraceScope t32("jacobi_fp32", 0.0, 0.0, c2.st);
        CK(jacobi32_precondition(R, ldr, w, Q, 8, c2.st));
    }
    for (int it = 0; it < 2; ++it) {
        CK(gemm(c2, "svd_precond", true, false, w, w, w, 1.0, Q, w, Q, w, 0.0, G, w));
        CK(copy_matrix(Q, w, Q1, w, w, w, c2.st));
        CK(gemm(c2, "svd_precond", false, false, w, w, w, -0.5, Q, w, G, w, 1.5, Q1, w));
        std::swap(Q, Q1);
    }
    CK(triu_copy(R, ldr, w, Ru, c2.st));
    CK(gemm(c2, "svd_precond", false, false, w, w, w, 1.0, Ru, w, Q, w, 0.0, X, w));
    TraceScope t64("jacobi_fp64", 0.0, 0.0, c2.st);
    CK(jacobi_svd(X, w, w, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status, sweep_cap(),
                  c2.st, true, true, Q));
    return cudaEventRecord(ss->svd_done, c2.st);
}

// Applies the pending step's Us, Vs on the side stream once the main stream
// has reached this point (after the next right update), then signals.
cudaError_t flush_pending(Ctx& c) {
    if (c.pending < 0) return cudaSuccess;
    SideStream* ss = nullptr;
    CK(side_stream(&ss));
    CK(cudaEventRecord(ss->right, c.st));
    CK(cudaStreamWaitEvent(ss->st, ss->right, 0));
    Ctx c2 = side_ctx(c, ss->st);
    Ctx::Step& rec = c.steps[(size_t)c.pending];
    const int64_t k0 = rec.k0, m = c.m, n = c.n, ldt = c.ldt;
    const int w = rec.w;
    double* T = c.T;
    if (k0 > 0) {  // T(0:k0, blk) := T(0:k0, blk) Vs
        CK(gemm(c2, "gemm_svdapply", false, false, k0, w, w, 1.0, T + k0 * ldt, ldt, c.w.Vs, w, 0.0, c2.w.tmp, k0));
        CK(copy_matrix(c2.w.tmp, k0, T + k0 * ldt, ldt, k0, w, c2.st));
    }
    const int64_t nr = n - k0 - w;
    if (nr > 0) {  // T(blk, k0+w:n) := Us^T T(blk, k0+w:n)
        CK(gemm(c2, "gemm_svdapply", true, false, w, nr, w, 1.0, c.w.Us, w, T + k0 + (k0 + w) * ldt, ldt, 0.0,
                c2.w.tmp, w));
        CK(copy_matrix(c2.w.tmp, w, T + k0 + (k0 + w) * ldt, ldt, w, nr, c2.st));
    }
    CK(set_diag_block(T, ldt, k0, m, w, c.w.D, c2.st));
    if (c.V) CK(defer_put(c, c.w.Vs, w, w, w, &rec.vs, c2.st));
    if (c.U) CK(defer_put(c, c.w.Us, w, w, w, &rec.us, c2.st));
    CK(cudaEventRecord(ss->applied, c2.st));
    c.pending = -1;
    c.applied_pending = true;
    return cudaSuccess;
}

// The main stream waits for the last queued application of a small SVD.
cudaError_t wait_applied(Ctx& c) {
    if (!c.applied_pending) return cudaSuccess;
    SideStream* ss = nullptr;
    CK(side_stream(&ss));
    CK(cudaStreamWaitEvent(c.st, ss->applied, 0));
    c.applied_pending = false;
    return cudaSuccess;
}

// Left update of a sketch step from the column split of T22 that the sketch
// made before the right update (emulated products, small SVD on the side
// stream).  With X2 = T(:, k0:n) W_V T_V and W_V = [W_1; W_2] (first b rows:
// the panel's columns), the right-updated trailing block is
// T22' = T22 - X2_b W_2^T (X2_b = X2(k0:m, :)), so the left update's
// W_U^T T22' = (T22^T W_U - W_2 (W_U^T X2_b)^T)^T: the large product reads
// the existing split of T22 instead of splitting T22' afresh, and only two
// small products are added.  Both terms are separate products with their
// own scales; the difference carries the absolute error of the right
// update itself (a few units of rounding of T22).  Call before the right
// update: it records the split and keeps W_2, which the panel QR overwrites.
cudaError_t left_from_old_split_prepare(Ctx& c, int64_t k0) {
    c.left_old = false;
    const int64_t mp = c.m - k0, np = c.n - k0, nt = np - c.b;
    if (!c.overlap || !emulated_prec(c.prec) || c.w.W2 == nullptr || nt < 16 || !oz_shape(c, np, c.b, mp))
        return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const OzOperand* ac = oz_cols_of(c, k0, &e);
    CK(e);
    c.left_cols = *ac;
    CK(copy_matrix(c.w.W + c.b, np, c.w.W2, nt, nt, c.b, c.st));
    c.left_old = true;
    return cudaSuccess;
}

// T22' := Q_U^T T22' on T(k0:m, k0+w:n) by the formula above (W_U, T_U in
// c.w.W, c.w.Tf; X2 in c.w.X2 from the right update).
cudaError_t apply_left_old(Ctx& c, int64_t k0, int w) {
    const int64_t m = c.m, mp = m - k0, nt = c.n - k0 - w, ldt = c.ldt;
    if (nt <= 0 || mp <= 0) return cudaSuccess;
    double* Y1 = c.w.G;  // nt x w
    CK(oz_cached_product(c, "gemm_left", c.left_cols, w, nt, w, c.w.W, mp, Y1, nt));
    CK(gemm(c, "gemm_left", true, false, w, w, mp, 1.0, c.w.W, mp, c.w.X2 + k0, m, 0.0, c.w.gram, w));
    CK(gemm(c, "gemm_left_tf", false, true, nt, w, w, -1.0, c.w.W2, nt, c.w.gram, w, 1.0, Y1, nt));
    CK(gemm(c, "gemm_left_tf", false, false, nt, w, w, 1.0, Y1, nt, c.w.Tf, w, 0.0, c.w.X, nt));
    return gemm(c, "gemm_left", false, true, mp, nt, w, -1.0, c.w.W, mp, c.w.X, nt, 1.0, c.T + k0 + (k0 + w) * ldt,
                ldt);
}

// Panel QR of T(k0:m, k0:k0+w), left update, small SVD and its application.
cudaError_t panel_and_svd(Ctx& c, int64_t k0, int w) {
    const int64_t m = c.m, n = c.n, ldt = c.ldt;
    const int64_t mp = m - k0;
    double* T = c.T;
    double* P = T + k0 + k0 * ldt;
    CK(factor_panel(c, P, ldt, mp, w));
    if (c.mode != MODE_FIXED)  // the learned-q features of the next step read this panel's R diagonal
        CK(copy_matrix(P, ldt + 1, c.w.rdiag, 1, 1, w, c.st));
    if (c.steps.empty() || c.steps.back().k0 != k0) c.steps.push_back(Ctx::Step{k0, w, false, 0, 0, 0, 0, 0, 0});
    c.steps.back().w = w;
    if (c.overlap) {
        // a sketch step flushed its predecessor after its right update; the
        // final block has none, so the previous step is applied here
        CK(flush_pending(c));
        CK(svd_side(c, P, ldt, w));
        c.pending = (int64_t)c.steps.size() - 1;
        if (c.left_old && w == c.b)
            CK(apply_left_old(c, k0, w));
        else
            CK(apply_left_t(c, T + k0 + (k0 + w) * ldt, ldt, mp, n - k0 - w, w));
        c.left_old = false;
        Ctx::Step& rec = c.steps.back();
        if (c.U) {  // U is accumulated backwards at the end from W_U, T_U, U_s
            CK(defer_put(c, c.w.W, mp, mp, w, &rec.wu));
            CK(defer_put(c, c.w.Tf, w, w, w, &rec.tu));
        }
        return cudaSuccess;  // applied after the next right update (flush_pending)
    }
    bool pre = false;
    CK(svd_block_begin(c, P, ldt, w, &pre));
    CK(apply_left_t(c, T + k0 + (k0 + w) * ldt, ldt, mp, n - k0 - w, w));
    Ctx::Step& rec = c.steps.back();
    if (c.U) {  // U is accumulated backwards at the end from W_U, T_U, U_s
        CK(defer_put(c, c.w.W, mp, mp, w, &rec.wu));
        CK(defer_put(c, c.w.Tf, w, w, w, &rec.tu));
    }
    CK(svd_block(c, P, ldt, w, pre));
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
    if (c.V) CK(defer_put(c, c.w.Vs, w, w, w, &rec.vs));
    if (c.U) CK(defer_put(c, c.w.Us, w, w, w, &rec.us));
    return cudaSuccess;
}

// X (len x cols, ld ldx) := (I - W Tf W^T) X with W (len x w, ld len) and
// the upper triangular Tf (w x w) of a compact WY product Q = I - W Tf W^T.
// Xs, X2s: w x cols scratch (default c.w.X, c.w.X2).
cudaError_t apply_left(Ctx& c, const double* W, const double* Tf, double* X, int64_t ldx, int64_t len, int64_t cols,
                       int w, double* Xs = nullptr, double* X2s = nullptr) {
    if (len <= 0 || cols <= 0) return cudaSuccess;
    if (!Xs) Xs = c.w.X;
    if (!X2s) X2s = c.w.X2;
    CK(gemm(c, "gemm_accumulate", true, false, w, cols, len, 1.0, W, len, X, ldx, 0.0, Xs, w));
    CK(gemm(c, "gemm_accumulate_tf", false, false, w, cols, w, 1.0, Tf, w, Xs, w, 0.0, X2s, w));
    return gemm(c, "gemm_accumulate", false, false, len, cols, w, -1.0, W, len, X2s, w, 1.0, X, ldx);
}

// Grouped form of the deferred accumulation (emulated products only).  An
// emulated product with K = b spends most of its time in the drain and the
// FP64 epilogue, once per output element and product, rather than in the
// MMAs.  The compact WY forms of up to kAccGroup consecutive steps are
// therefore merged into one, Q_i Q_{i+1} ... = I - W T W^T with
// W = [W_i, W_{i+1}, ...] (each W_j placed at its own first row k0_j - k0_i)
// and T built step by step by the block rule of a product of two compact WY
// forms, T = [[T_a, -T_a (W_a^T W_b) T_b], [0, T_b]] (Sec. 2.3): one update
// with K = kAccGroup b replaces kAccGroup updates with K = b.  The group's
// S factors act on its own diagonal blocks, which the later Q's of the group
// do not touch, so they commute with those Q's and are written first.  The
// scratch is carved from the cached-split buffer, unused once the
// factorization loop has ended; the merges run on the side stream.
constexpr int kAccGroup = 4;

struct AccScratch {
    double *Wb[2], *Tb[2];  // merged W and T, one per group in flight
    double *G, *Y, *X, *X2;
    void* oz;               // emulated-product work of the merges (side stream)
    size_t oz_bytes;
};

bool acc_scratch(Ctx& c, int64_t nx, AccScratch* sc) {
    if (!emulated_prec(c.prec) || c.w.oz_rows == nullptr) return false;
    const size_t wg = (size_t)kAccGroup * c.b;
    // the merges' own emulated-product work: two split operands of up to
    // wg x nx and the split-K partials of a wg x wg product
    const size_t ozb = 2 * oz_operand_bytes((int64_t)wg, nx) + sizeof(double) * wg * wg * 64 + 4096;
    const size_t need = align_up(sizeof(double) * (size_t)nx * wg) * 4 + 3 * align_up(sizeof(double) * wg * wg) +
                        align_up(sizeof(double) * wg * (size_t)c.b) + align_up(ozb);
    if (need > c.w.oz_rows_bytes) return false;
    char* p = (char*)c.w.oz_rows;
    auto take = [&](size_t elems) {
        double* q = (double*)p;
        p += align_up(sizeof(double) * elems);
        return q;
    };
    sc->Wb[0] = take((size_t)nx * wg);
    sc->Wb[1] = take((size_t)nx * wg);
    sc->X = take((size_t)nx * wg);
    sc->X2 = take((size_t)nx * wg);
    sc->Tb[0] = take(wg * wg);
    sc->Tb[1] = take(wg * wg);
    sc->G = take(wg * wg);
    sc->Y = take(wg * (size_t)c.b);
    sc->oz = (void*)p;
    sc->oz_bytes = ozb;
    c.oc = OzCache{-1};  // the cached splits are overwritten from here on
    return true;
}

// Merged W (len0 x wsum, ld len0) and T (wsum x wsum, ld wsum) of steps
// i0..i1 (consecutive, each with a transform) of the U (is_v false) or V
// factor, into Wm, Tm; k0 of step i0 is the group's first row.  Every block
// W_a^T W_b the rule needs comes from one product,
// W(:, 0:wsum-w_last)^T W(:, w_0:wsum) (its lower blocks are not used).
// c supplies the steps and the deferred store, cx the stream and the work
// buffers of the products (the side stream's, when the merge runs there).
cudaError_t merge_wy(const Ctx& c, Ctx& cx, double* Wm, double* Tm, double* Gs, double* Ys, int64_t nx, bool is_v,
                     int64_t i0, int64_t i1, int* wsum_out) {
    const int64_t k00 = c.steps[(size_t)i0].k0, len0 = nx - k00;
    auto width = [&](int64_t j) { return is_v ? c.b : c.steps[(size_t)j].w; };
    int wsum = 0;
    for (int64_t j = i0; j <= i1; ++j) wsum += width(j);
    const int w0 = width(i0), wl = width(i1);
    TraceScope ts("gemm_accumulate_merge", 0.0, 8.0 * (double)len0 * wsum, cx.st);
    CK(cudaMemsetAsync(Wm, 0, sizeof(double) * (size_t)len0 * wsum, cx.st));
    CK(cudaMemsetAsync(Tm, 0, sizeof(double) * (size_t)wsum * wsum, cx.st));
    int off = 0;
    for (int64_t j = i0; j <= i1; ++j) {
        const Ctx::Step& r = c.steps[(size_t)j];
        const int wj = width(j);
        const int64_t lenj = nx - r.k0;
        CK(copy_matrix(c.w.defer + (is_v ? r.wv : r.wu), lenj, Wm + (r.k0 - k00) + (int64_t)off * len0, len0, lenj,
                       wj, cx.st));
        CK(copy_matrix(c.w.defer + (is_v ? r.tv : r.tu), wj, Tm + off + (int64_t)off * wsum, wsum, wj, wj, cx.st));
        off += wj;
    }
    // Gc (wsum - wl) x (wsum - w0), ld wsum - wl: block (a, b) = W_a^T W_b
    const int gr = wsum - wl, gc = wsum - w0;
    CK(gemm(cx, "gemm_accumulate_merge", true, false, gr, gc, len0, 1.0, Wm, len0, Wm + (int64_t)w0 * len0, len0,
            0.0, Gs, gr));
    int wacc = w0;
    for (int64_t j = i0 + 1; j <= i1; ++j) {  // T(0:wacc, wacc:wacc+wj) = -T_acc (W_acc^T W_j) T_j
        const int wj = width(j);
        const double* Gj = Gs + (int64_t)(wacc - w0) * gr;  // rows 0:wacc of the column block of step j
        CK(gemm(cx, "gemm_accumulate_merge", false, false, wacc, wj, wacc, 1.0, Tm, wsum, Gj, gr, 0.0, Ys, wacc));
        CK(gemm(cx, "gemm_accumulate_merge", false, false, wacc, wj, wj, -1.0, Ys, wacc, Tm + wacc + (int64_t)wacc * wsum,
                wsum, 0.0, Tm + (int64_t)wacc * wsum, wsum));
        wacc += wj;
    }
    *wsum_out = wsum;
    return cudaSuccess;
}

// Deferred accumulation of the orthogonal factors (the backward order of
// LAPACK's dorgqr).  With Q_i = I - W_i Tf_i W_i^T acting on indices >= k0_i
// and S_i = diag(I, s_i, I) the small-SVD factor at block i,
//   V = Q_0 S_0 Q_1 S_1 ... ,  so  X := I;  for i = last..0: X := Q_i (S_i X).
// Before step i, X differs from I only in rows and columns >= k0_i + w_i, so
// S_i X just writes s_i into the diagonal block and Q_i touches X(k0_i:, k0_i:)
// only: (n - k0_i)^2 instead of n (n - k0_i) per step, a third less work than
// updating V at every step.
cudaError_t accumulate(Ctx& c, double* X, int64_t nx, int64_t ldx, bool is_v) {
    CK(set_identity(X, nx, ldx, c.st));
    AccScratch sc{};
    const bool grouped = acc_scratch(c, nx, &sc);
    auto has_q = [&](int64_t j) { return !is_v || c.steps[(size_t)j].sketch; };
    struct Grp {
        int64_t i0, i1;
    };
    std::vector<Grp> groups;  // from the last step back
    for (int64_t i = (int64_t)c.steps.size() - 1; i >= 0;) {
        int64_t i0 = i;
        if (grouped && has_q(i))
            while (i0 > 0 && i - i0 + 1 < kAccGroup && has_q(i0 - 1)) --i0;
        groups.push_back(Grp{i0, i});
        i = i0 - 1;
    }
    // The merges run on the side stream one group ahead of the updates, each
    // into one of two buffers: the merge of the next group overlaps the
    // update of this one.  The side stream first waits for everything the
    // main stream has queued (the deferred store is complete).
    std::vector<size_t> merged_groups;
    for (size_t k = 0; k < groups.size(); ++k)
        if (groups[k].i1 > groups[k].i0) merged_groups.push_back(k);
    SideStream* ss = nullptr;
    Ctx c2;
    std::vector<int> wsums(groups.size(), 0);
    auto launch_merge = [&](size_t t) -> cudaError_t {  // t-th merged group, buffer t % 2
        const Grp& g = groups[merged_groups[t]];
        const int bsel = (int)(t % 2);
        CK(cudaStreamWaitEvent(ss->st, ss->freed[bsel], 0));  // no wait before the buffer's first use
        CK(merge_wy(c, c2, sc.Wb[bsel], sc.Tb[bsel], sc.G, sc.Y, nx, is_v, g.i0, g.i1, &wsums[merged_groups[t]]));
        return cudaEventRecord(ss->merged[bsel], ss->st);
    };
    if (!merged_groups.empty()) {
        CK(side_stream(&ss));
        c2 = side_ctx(c, ss->st);
        c2.w.oz = sc.oz;
        c2.w.oz_bytes = sc.oz_bytes;
        CK(cudaEventRecord(ss->right, c.st));
        CK(cudaStreamWaitEvent(ss->st, ss->right, 0));
        CK(launch_merge(0));
    }
    size_t t = 0;  // merged groups applied so far
    for (size_t k = 0; k < groups.size(); ++k) {
        const Grp& g = groups[k];
        for (int64_t j = g.i1; j >= g.i0; --j) {
            const Ctx::Step& r = c.steps[(size_t)j];
            CK(copy_matrix(c.w.defer + (is_v ? r.vs : r.us), r.w, X + r.k0 + r.k0 * ldx, ldx, r.w, r.w, c.st));
        }
        const Ctx::Step& r0 = c.steps[(size_t)g.i0];
        double* Xb = X + r0.k0 + r0.k0 * ldx;
        if (!has_q(g.i1)) {
        } else if (g.i0 == g.i1) {
            const int w = is_v ? c.b : r0.w;
            CK(apply_left(c, c.w.defer + (is_v ? r0.wv : r0.wu), c.w.defer + (is_v ? r0.tv : r0.tu), Xb, ldx,
                          nx - r0.k0, nx - r0.k0, w));
        } else {
            if (t + 1 < merged_groups.size()) CK(launch_merge(t + 1));
            const int bsel = (int)(t % 2);
            CK(cudaStreamWaitEvent(c.st, ss->merged[bsel], 0));
            CK(apply_left(c, sc.Wb[bsel], sc.Tb[bsel], Xb, ldx, nx - r0.k0, nx - r0.k0, wsums[k], sc.X, sc.X2));
            CK(cudaEventRecord(ss->freed[bsel], c.st));
            ++t;
        }
    }
    return cudaSuccess;
}

// C (rows x cols) := C (I - W Tf W^T) with W (cols x w, ld cols) and Tf (w x w).
cudaError_t apply_right_wy(Ctx& c, double* C, int64_t ldc, int64_t rows, int64_t cols, const double* W,
                           const double* Tf, int w) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    CK(gemm(c, "gemm_accumulate", false, false, rows, w, cols, 1.0, C, ldc, W, cols, 0.0, c.w.X, rows));
    CK(gemm(c, "gemm_accumulate_tf", false, false, rows, w, w, 1.0, c.w.X, rows, Tf, w, 0.0, c.w.X2, rows));
    return gemm(c, "gemm_accumulate", false, true, rows, cols, w, -1.0, c.w.X2, rows, W, cols, 1.0, C, ldc);
}

// Forward accumulation into orthogonal factors that already hold a partial
// factorization (resume): with the new steps' Q_i = I - W_i Tf_i W_i^T on
// columns k0_i.. and S_i on the block columns, X := X Q_i S_i for each new
// step in order (the per-step updates of the paper's loop).
cudaError_t accumulate_forward(Ctx& c, double* X, int64_t nx, int64_t ldx, bool is_v) {
    for (const Ctx::Step& r : c.steps) {
        double* Xc = X + r.k0 * ldx;
        if (!is_v || r.sketch) {
            const int w = is_v ? c.b : r.w;
            CK(apply_right_wy(c, Xc, ldx, nx, nx - r.k0, c.w.defer + (is_v ? r.wv : r.wu),
                              c.w.defer + (is_v ? r.tv : r.tu), w));
        }
        CK(gemm(c, "gemm_accumulate", false, false, nx, r.w, r.w, 1.0, Xc, ldx, c.w.defer + (is_v ? r.vs : r.us),
                r.w, 0.0, c.w.tmp, nx));
        CK(copy_matrix(c.w.tmp, nx, Xc, ldx, nx, r.w, c.st));
    }
    return cudaSuccess;
}

// Y = (T22^T T22)^q T22^T G with 16-bit operands on tcgen05 (FP32 accumulate)
// and FP32 shifted-CholeskyQR re-orthonormalisation after every product but
// the last.  lowp_begin leaves Y0 = T22^T G in c.w.Xf (FP32); lowp_iterate
// applies `iters` power-iteration pairs to it; lowp_finish copies the result
// to FP64 in c.w.Y (n' x b).
struct LowpShape {
    int64_t mp, np, lds, ldst;
    int npad;
    bool f16;
};

LowpShape lowp_shape(const Ctx& c, int64_t mp, int64_t np) {
    return LowpShape{mp, np, round8(mp), round8(np), tc_gemm_npad(c.b), c.prec == RANDUTV_SKETCH_FP16_SCALED};
}

// (A, lda, M, K) = (S, lds, n', m') for T22^T X; (St, ldst, m', n') for T22 X
cudaError_t lowp_product(Ctx& c, const LowpShape& s, bool transposed, int64_t ldb) {
    const int b = c.b;
    const uint16_t* A = transposed ? c.w.S : c.w.St;
    const int64_t lda = transposed ? s.lds : s.ldst;
    const int64_t M = transposed ? s.np : s.mp, K = transposed ? s.mp : s.np;
    const int splits = tc_gemm_splits(M, K, c.sms);
    {
        TraceScope ts("tc_gemm_sketch", 2.0 * (double)M * b * K,
                      2.0 * ((double)M * K + (double)b * K) + 4.0 * splits * (double)M * s.npad, c.st);
        CK(tc_gemm(A, lda, c.w.B16, ldb, M, b, K, s.f16, c.w.Pf, M, M * s.npad, splits, c.w.status, c.st));
    }
    TraceScope ts("lowp_reduce", 0.0, 4.0 * (splits + 1.0) * (double)M * b, c.st);
    return reduce_splits(c.w.Pf, M * s.npad, splits, M, b, M, c.w.Xf, c.st);
}

cudaError_t lowp_begin(Ctx& c, int64_t i, const double* T22, const LowpShape& s) {
    const int b = c.b;
    {
        TraceScope ts("lowp_shadow", 0.0, (8.0 + 4.0) * (double)s.mp * s.np, c.st);
        if (s.f16) CK(absmax_f64(T22, c.ldt, s.mp, s.np, c.w.amax, c.st));
        CK(shadow16(T22, c.ldt, s.mp, s.np, c.w.S, s.lds, c.w.St, s.ldst, s.f16, c.w.amax, c.st));
    }
    {
        TraceScope ts("gaussian", 0.0, 8.0 * (double)s.mp * b, c.st);
        CK(gaussian_f64(c.seed, i, s.mp, b, c.w.G, s.mp, c.st));
        CK(pack16_f64(c.w.G, s.mp, s.mp, b, c.w.B16, s.lds, s.f16, c.st));
    }
    return lowp_product(c, s, true, s.lds);  // Y0 = T22^T G
}

cudaError_t lowp_iterate(Ctx& c, const LowpShape& s, int iters) {
    for (int it = 0; it < iters; ++it) {
        {
            TraceScope ts("lowp_cholqr", 0.0, 0.0, c.st);
            CK(cholqr32(c.w.Xf, s.np, c.b, 3, c.w.B16, s.ldst, s.f16, c.w.cqr, c.sms, c.st));
        }
        CK(lowp_product(c, s, false, s.ldst));  // Z = T22 Y
        {
            TraceScope ts("lowp_cholqr", 0.0, 0.0, c.st);
            CK(cholqr32(c.w.Xf, s.mp, c.b, 3, c.w.B16, s.lds, s.f16, c.w.cqr, c.sms, c.st));
        }
        CK(lowp_product(c, s, true, s.lds));  // Y = T22^T Z
    }
    return cudaSuccess;
}

cudaError_t lowp_finish(Ctx& c, const LowpShape& s) { return f32_to_f64(c.w.Xf, s.np * c.b, c.w.Y, c.st); }

// FP64 sketch of T22 = T(k0:m, k0:n): Y0 = T22^T G into c.w.Y; iterate:
// Y := T22^T (T22 Y).
cudaError_t fp64_begin(Ctx& c, int64_t i, int64_t k0) {
    const int64_t mp = c.m - k0, np = c.n - k0;
    {
        TraceScope ts("gaussian", 0.0, 8.0 * (double)mp * c.b, c.st);
        CK(gaussian_f64(c.seed, i, mp, c.b, c.w.G, mp, c.st));
    }
    return sketch_gemm(c, true, k0, c.w.G, mp, c.w.Y, np);
}

cudaError_t fp64_iterate(Ctx& c, int64_t k0, double* Y, int iters) {
    const int64_t mp = c.m - k0, np = c.n - k0;
    for (int it = 0; it < iters; ++it) {
        CK(sketch_gemm(c, false, k0, Y, np, c.w.Z, mp));
        CK(sketch_gemm(c, true, k0, c.w.Z, mp, Y, np));
    }
    return cudaSuccess;
}

// Added to the step index in the key of the CountSketch signs of the features.
constexpr int64_t kFeatureDrawStep = (int64_t)1 << 40;

// Features of block step i (needs Y0 = T22^T G in c.w.Y): the Householder R
// of E = S Y0 (2b x b, S the structured CountSketch r -> r mod 2b with random
// signs; E = Y0 when n' <= 2b), in FP32 in one block for b <= 128, and the
// previous block's R diagonal (from its panel QR), read from dprev[j * dstride].
cudaError_t block_features(Ctx& c, int64_t i, int64_t np, const double* dprev, int64_t dstride) {
    const int b = c.b;
    TraceScope ts("learnq_features", 0.0, 8.0 * (double)np * b, c.st);
    const int64_t e = std::min<int64_t>(2 * (int64_t)b, np);
    double* E = c.w.X2;  // e x b, ld e
    if (np <= 2 * (int64_t)b)
        CK(copy_matrix(c.w.Y, np, E, e, np, b, c.st));
    else
        CK(countsketch(c.w.Y, np, np, b, (int)e, c.seed ^ (uint64_t)(kFeatureDrawStep + i), E, c.st));
    if (e <= 256 && b <= 128) {  // |R_jj| of E by a one-block FP32 QR
        CK(feature_rdiag(E, e, e, b, c.w.sdiag, c.w.level, c.st));
        return learnq_features(dprev, dstride, dprev ? b : 0, c.w.sdiag, 0, b, c.w.feat, c.w.level, true, c.st);
    }
    CK(panel_qr(E, e, e, b, c.w.tau, c.w.pscr, c.w.bars, c.w.status, panel_sms(c), c.st));
    return learnq_features(dprev, dstride, dprev ? b : 0, E, e, b, c.w.feat, c.w.level, false, c.st);
}

// The cached splits of T(:, k0:n) (rows) and T22 (columns), made now, outside
// any launch gate, so that the host's record of them is always true.
cudaError_t prefetch_splits(Ctx& c, int64_t k0) {
    const int64_t mp = c.m - k0, np = c.n - k0;
    cudaError_t e = cudaSuccess;
    if (oz_shape(c, np, c.b, mp)) {
        oz_cols_of(c, k0, &e);
        CK(e);
    }
    if (oz_shape(c, mp, c.b, np)) {
        oz_rows_of(c, k0, &e);
        CK(e);
    }
    return cudaSuccess;
}

// Trace mode: diagonal the step would produce with q = 0..3, i.e. the
// singular values of T22 Q1(q), Q1(q) = orth((T22^T T22)^q Y0); the q = 2
// sketch is left in c.w.Y for the step itself.
cudaError_t trace_candidates(Ctx& c, int64_t k0) {
    const int64_t mp = c.m - k0, np = c.n - k0;
    const int b = c.b;
    double* Yc = c.w.tmp;
    CK(copy_matrix(c.w.Y, np, Yc, np, np, b, c.st));
    for (int q = 0; q < 4; ++q) {
        if (q > 0) CK(fp64_iterate(c, k0, Yc, 1));
        if (q == 2) CK(copy_matrix(Yc, np, c.w.Y, np, np, b, c.st));
        // explicit Q1 of the Householder QR of Yc
        CK(copy_matrix(Yc, np, c.w.X2, np, np, b, c.st));
        CK(factor_panel(c, c.w.X2, np, np, b));
        CK(set_eye_rect(c.w.X, np, b, np, c.st));
        CK(gemm(c, "learnq_trace", false, true, b, b, b, 1.0, c.w.Tf, b, c.w.W, np, 0.0, c.w.G, b));
        CK(gemm(c, "learnq_trace", false, false, np, b, b, -1.0, c.w.W, np, c.w.G, b, 1.0, c.w.X, np));
        // sigma(T22 Q1) from the R of its QR
        CK(sketch_gemm(c, false, k0, c.w.X, np, c.w.Z, mp));
        CK(panel_qr(c.w.Z, mp, mp, b, c.w.tau, c.w.pscr, c.w.bars, c.w.status, c.sms, c.st));
        CK(jacobi_svd(c.w.Z, mp, b, c.w.D, c.w.Us, c.w.Vs, c.w.jscr, c.w.bars + 1, c.w.counters, c.w.status,
                      sweep_cap(), c.st));
        CK(cudaMemcpyAsync(c.w.dq + (size_t)q * b, c.w.D, sizeof(double) * b, cudaMemcpyDeviceToDevice, c.st));
    }
    return cudaSuccess;
}

// One sketch step (n' > b) at column offset k0.
cudaError_t sketch_step(Ctx& c, int64_t i) {
    const int64_t m = c.m, n = c.n, ldt = c.ldt;
    const int b = c.b;
    const int64_t k0 = i * (int64_t)b, mp = m - k0, np = n - k0;
    double* T22 = c.T + k0 + k0 * ldt;
    // the 16-bit tensor-core sketch needs b % 16 == 0, b <= 256 and a trailing
    // matrix of at least 128 x 128 (one TMA box); smaller steps stay in FP64
    const bool lowp = lowp_prec(c.prec) && b % 16 == 0 && b <= 256 && mp >= 128 && np >= 128;
    const LowpShape ls = lowp_shape(c, mp, np);
    int iters = c.q;
    CK(wait_applied(c));  // the previous application must reach T before its rows are split
    if (c.mode == MODE_FIXED) {
        if (lowp) {
            CK(lowp_begin(c, i, T22, ls));
            CK(lowp_iterate(c, ls, iters));
            CK(lowp_finish(c, ls));
        } else {
            CK(fp64_begin(c, i, k0));
            CK(fp64_iterate(c, k0, c.w.Y, iters));
        }
    } else if (c.mode == MODE_TRACE && i > 0 && (i % c.tr_stride != c.tr_offset || c.tr_count >= c.tr_max)) {
        CK(fp64_begin(c, i, k0));  // a step that is not recorded: the q = 2 trajectory itself
        CK(fp64_iterate(c, k0, c.w.Y, 2));
    } else if (c.mode == MODE_TRACE) {
        CK(fp64_begin(c, i, k0));
        CK(block_features(c, i, np, i > c.start_step ? c.w.rdiag : nullptr, 1));
        CK(trace_candidates(c, k0));
        if (c.tr_count < c.tr_max) {
            double cand[4 * 512];
            CK(cudaMemcpyAsync(c.tr_feat + 16 * c.tr_count, c.w.feat, sizeof(float) * 16, cudaMemcpyDeviceToHost,
                               c.st));
            CK(cudaMemcpyAsync(cand, c.w.dq, sizeof(double) * 4 * b, cudaMemcpyDeviceToHost, c.st));
            CK(cudaStreamSynchronize(c.st));
            // label: smallest q whose diagonal is within 5% of the q = 2 one;
            // entries below 1e-13 of the largest singular value estimate (the
            // first block's first entry) are rounding noise and are skipped,
            // so a block made only of noise is labelled 0
            if (i == 0) c.t00 = cand[2 * b];
            const double floor_ = 1e-13 * std::max(c.t00, cand[2 * b]);
            int label = 2;
            for (int q = 0; q < 2; ++q) {
                double worst = 0.0;
                for (int j = 0; j < b; ++j) {
                    double ref = cand[2 * b + j];
                    if (!(ref > floor_)) continue;
                    worst = std::max(worst, std::fabs(cand[q * b + j] / ref - 1.0));
                }
                if (worst <= 0.05) {
                    label = q;
                    break;
                }
            }
            c.tr_label[c.tr_count] = label;
            if (c.tr_cand)
                for (int e = 0; e < 4 * b; ++e) c.tr_cand[(size_t)c.tr_count * 4 * b + e] = cand[e];
            ++c.tr_count;
        }
    } else {  // MODE_LEARNED: q is chosen and applied on the device
        if (lowp) {
            CK(lowp_begin(c, i, T22, ls));
            CK(lowp_finish(c, ls));
        } else {
            CK(fp64_begin(c, i, k0));
        }
        // the previous block's decay: the R diagonal of its panel QR, ready
        // before its small SVD (which keeps overlapping this step)
        CK(block_features(c, i, np, i > c.start_step ? c.w.rdiag : nullptr, 1));
        CK(learnq_infer(c.have_model ? c.w.qmodel : nullptr, c.w.feat, c.q, c.w.qdev, c.w.qlog + i, c.st));
        if (!lowp) CK(prefetch_splits(c, k0));
        // every iteration up to q = 3 is queued; the kernels of iteration it
        // run only when the chosen q (device) is at least it + 1
        for (int it = 0; it < 3; ++it) {
            GateScope gate(c.w.qdev, it + 1);
            if (lowp)
                CK(lowp_iterate(c, ls, 1));
            else
                CK(fp64_iterate(c, k0, c.w.Y, 1));
        }
        if (lowp) CK(lowp_finish(c, ls));
    }
    CK(factor_panel(c, c.w.Y, np, np, b));
    CK(left_from_old_split_prepare(c, k0));
    CK(apply_right_T(c, k0, b));
    CK(flush_pending(c));  // the previous step's Us^T may now reach rows blk_{i-1}
    Ctx::Step rec{k0, b, true, 0, 0, 0, 0, 0, 0};
    if (c.V) {  // V is accumulated backwards at the end from W_V, T_V, V_s
        CK(defer_put(c, c.w.W, np, np, b, &rec.wv));
        CK(defer_put(c, c.w.Tf, b, b, b, &rec.tv));
    }
    c.steps.push_back(rec);
    return panel_and_svd(c, k0, b);
}

// Tolerance stop (Sec. 1.1: stop once the rank is revealed): the host reads
// the diagonal D of the block step just queued (on the stream its SVD runs
// on) and stops after the first block whose smallest entry is at most
// rank_tol |T_00|.
cudaError_t tol_check(Ctx& c, int64_t k0, int w, bool* stop) {
    *stop = false;
    c.dhost.assign((size_t)w, 0.0);
    cudaStream_t st = c.st;
    if (c.overlap) {
        SideStream* ss = nullptr;
        CK(side_stream(&ss));
        st = ss->st;
    }
    CK(cudaMemcpyAsync(c.dhost.data(), c.w.D, sizeof(double) * (size_t)w, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (k0 == 0) c.t00 = std::fabs(c.dhost[0]);
    const double thr = c.rank_tol * c.t00;
    for (int j = 0; j < w; ++j)
        if (std::fabs(c.dhost[(size_t)j]) > thr) ++c.rank;
    *stop = !(std::fabs(c.dhost[(size_t)w - 1]) > thr);
    return cudaSuccess;
}

cudaError_t run_factor(Ctx& c, const double* A, int64_t lda, int64_t stop_after) {
    const int64_t m = c.m, n = c.n;
    if (!c.resume && A != c.T) CK(copy_matrix(A, lda, c.T, c.ldt, m, n, c.st));
    CK(check_finite(c.T, c.ldt, m, n, c.w.status, c.st));
    c.steps.clear();
    c.pending = -1;
    c.applied_pending = false;
    // the trace mode uses the SVD buffers itself and stays serial; the learned
    // mode reads the previous block's D as soon as its SVD is done
    c.overlap = (c.mode == MODE_FIXED || c.mode == MODE_LEARNED);
    c.cols_done = std::min<int64_t>(n, c.start_step * (int64_t)c.b);
    for (int64_t i = c.start_step;; ++i) {
        if (stop_after >= 0 && i - c.start_step >= stop_after) break;
        const int64_t k0 = i * (int64_t)c.b;
        const int64_t np = n - k0;
        if (np <= 0) break;
        const int w = (int)std::min<int64_t>(np, c.b);
        if (np <= c.b)
            CK(panel_and_svd(c, k0, w));
        else
            CK(sketch_step(c, i));
        c.cols_done = k0 + w;
        if (c.rank_tol > 0.0) {
            bool stop = false;
            CK(tol_check(c, k0, w, &stop));
            if (stop) break;
        }
        if (np <= c.b) break;
    }
    CK(flush_pending(c));
    CK(wait_applied(c));
    if (c.resume) {
        if (c.V) CK(accumulate_forward(c, c.V, n, c.ldv, true));
        if (c.U) CK(accumulate_forward(c, c.U, m, c.ldu, false));
    } else {
        if (c.V) CK(accumulate(c, c.V, n, c.ldv, true));
        if (c.U) CK(accumulate(c, c.U, m, c.ldu, false));
    }
    return cudaSuccess;
}

// randUTV with a QR first, for tall inputs (Sec. 5.1): blocked Householder QR
// A = Q_A [R; 0] (panels of b columns, each with its compact WY factor and a
// left update of the columns to its right), T := [R; 0], randUTV of the n x n
// R in place (its U_R lands in U(0:n, 0:n)), then U := Q_A diag(U_R, I) by
// applying the panels' reflectors from the left, last panel first.
cudaError_t run_qr_first(Ctx& c, const double* A, int64_t lda, int64_t stop_after) {
    const int64_t m = c.m, n = c.n, ldt = c.ldt;
    if (A != c.T) CK(copy_matrix(A, lda, c.T, ldt, m, n, c.st));
    CK(check_finite(c.T, ldt, m, n, c.w.status, c.st));
    c.qr.clear();
    c.overlap = false;
    for (int64_t k0 = 0; k0 < n; k0 += c.b) {
        const int w = (int)std::min<int64_t>(c.b, n - k0);
        const int64_t mp = m - k0;
        CK(factor_panel(c, c.T + k0 + k0 * ldt, ldt, mp, w));
        if (n - k0 - w > 0) CK(apply_left_t(c, c.T + k0 + (k0 + w) * ldt, ldt, mp, n - k0 - w, w));
        if (c.U) {
            Ctx::QrStep q{k0, w, 0, 0};
            CK(defer_put(c, c.w.W, mp, mp, w, &q.wu));
            CK(defer_put(c, c.w.Tf, w, w, w, &q.tu));
            c.qr.push_back(q);
        }
    }
    CK(zero_below_diag(c.T, ldt, m, n, c.st));
    c.m = n;  // randUTV of R = T(0:n, 0:n); rows n..m of T stay zero
    c.oc = OzCache{};
    const cudaError_t e = run_factor(c, c.T, ldt, stop_after);
    c.m = m;
    c.oc = OzCache{};
    CK(e);
    if (c.U) {
        CK(embed_identity(c.U, c.ldu, m, n, c.st));
        for (auto it = c.qr.rbegin(); it != c.qr.rend(); ++it)
            CK(apply_left(c, c.w.defer + it->wu, c.w.defer + it->tu, c.U + it->k0, c.ldu, m - it->k0, m, it->w));
    }
    return cudaSuccess;
}

// A wait that gave up leaves the kernels after it working on partial data,
// which may then also raise the other flags, so a timeout is reported first.
randutv_status status_from_bits(int bits) {
    if (bits & ST_TIMEOUT) return RANDUTV_ETIMEOUT;
    if (bits & ST_NONFINITE) return RANDUTV_ENONFINITE;
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

void randutv_set_limits(int64_t wait_polls, int max_sweeps) {
    g_wait_limit.store(wait_polls > 0 ? (long long)wait_polls : kSpinLimit, std::memory_order_relaxed);
    g_sweep_cap.store(max_sweeps > 0 ? max_sweeps : kDefaultSweeps, std::memory_order_relaxed);
}

size_t randutv_workspace_size(int64_t m, int64_t n, int b, int prec) {
    if (m < n || n < 0 || b < 1) return 0;
    if (!valid_prec(prec)) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return make_layout(m, n, b, device_sms(dev), prec).total;
}

}  // extern "C"

namespace rutv {
namespace {

// Options of randutv_factor_opt (see the header).
struct FactorOpts {
    int64_t start_col = 0;
    double rank_tol = 0.0;
    bool qr_first = false;
    int64_t* cols_done = nullptr;
    int64_t* rank = nullptr;
};

struct ModeArgs {
    int mode = MODE_FIXED;
    const float* model = nullptr;  // host parameters (learned mode)
    int* q_used = nullptr;
    float* tr_feat = nullptr;
    int* tr_label = nullptr;
    double* tr_cand = nullptr;
    int64_t tr_max = 0;
    int64_t* tr_count = nullptr;
    int64_t tr_stride = 1;
};

// The device address of page-locked host memory (registered or allocated by
// CUDA), or null for any other pointer.
const void* pinned_device_address(const void* host) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

randutv_status factor_impl(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed, double* U,
                           double* T, double* V, int prec, void* stream, void* workspace, size_t ws_bytes,
                           int64_t stop_after, int* info, const ModeArgs& ma, const FactorOpts& fo = FactorOpts{}) {
    if (!args_ok(m, n, A, lda, b, q, T)) return RANDUTV_EINVAL;
    if (!valid_prec(prec)) return RANDUTV_ENOTIMPL;
    if (A == T && lda != m) return RANDUTV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RANDUTV_ECUDA;
    const int sms = device_sms(dev);
    Layout L = make_layout(m, n, b, sms, prec, fo.qr_first);
    void* base = workspace;
    if (base == nullptr) {
        if (cached_workspace(dev, L.total, &base) != cudaSuccess) return RANDUTV_ENOMEM;
    } else if (ws_bytes < L.total) {
        return RANDUTV_ENOMEM;
    }
    Ctx c{};
    c.m = m; c.n = n; c.ldt = std::max<int64_t>(m, 1);
    c.b = b; c.q = q; c.seed = seed; c.prec = prec;
    c.U = U; c.T = T; c.V = V;
    c.w = carve(base, L);
    c.sms = sms;
    c.st = st;
    c.mode = ma.mode;
    c.tr_feat = ma.tr_feat;
    c.tr_label = ma.tr_label;
    c.tr_cand = ma.tr_cand;
    c.tr_max = ma.tr_max;
    c.tr_stride = std::max<int64_t>(ma.tr_stride, 1);
    c.tr_offset = (int64_t)(seed % (uint64_t)c.tr_stride);
    c.ldu = std::max<int64_t>(m, 1);
    c.ldv = std::max<int64_t>(n, 1);
    c.defer_top = 0;
    c.rank_tol = fo.rank_tol;
    if (fo.start_col > 0) {  // resume: steps continue at index start_col / b
        c.resume = true;
        c.start_step = fo.start_col / b;
        c.cols_done = fo.start_col;
        if (fo.rank_tol > 0.0) {  // T_00 and the rank so far from the diagonal already in T
            c.dhost.assign((size_t)fo.start_col, 0.0);
            if (cudaMemcpy2DAsync(c.dhost.data(), sizeof(double), T, sizeof(double) * (size_t)(c.ldt + 1),
                                  sizeof(double), (size_t)fo.start_col, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return RANDUTV_ECUDA;
            c.t00 = std::fabs(c.dhost[0]);
            for (double d : c.dhost)
                if (std::fabs(d) > fo.rank_tol * c.t00) ++c.rank;
        }
        if (fo.start_col >= n) {  // nothing left to factor
            if (fo.cols_done) *fo.cols_done = n;
            if (fo.rank) *fo.rank = c.rank_tol > 0.0 ? c.rank : n;
            return RANDUTV_OK;
        }
    }
    if (cudaMemsetAsync(c.w.status, 0, sizeof(int), st) != cudaSuccess) return RANDUTV_ECUDA;
    if (lowp_prec(prec)) {  // rows b..npad-1 of the 16-bit B operand stay zero
        size_t bytes = sizeof(uint16_t) * (size_t)tc_gemm_npad(std::min<int64_t>(b, std::max<int64_t>(n, 1))) *
                       round8(std::max<int64_t>(std::max(m, n), 1));
        if (cudaMemsetAsync(c.w.B16, 0, bytes, st) != cudaSuccess) return RANDUTV_ECUDA;
    }
    if (ma.mode == MODE_LEARNED && ma.model != nullptr) {
        if (cudaMemcpyAsync(c.w.qmodel, ma.model, sizeof(float) * learnq_nparam(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return RANDUTV_ECUDA;
        c.have_model = true;
    }
    const int64_t nblocks = (n + b - 1) / b;
    if (ma.q_used)
        for (int64_t i = 0; i < nblocks; ++i) ma.q_used[i] = -1;
    if (ma.mode == MODE_LEARNED && nblocks > 0 &&
        cudaMemsetAsync(c.w.qlog, 0xFF, sizeof(int) * (size_t)nblocks, st) != cudaSuccess)
        return RANDUTV_ECUDA;
    if (fo.cols_done) *fo.cols_done = c.cols_done;
    if (fo.rank) *fo.rank = c.rank_tol > 0.0 ? c.rank : c.cols_done;
    if (m == 0) return RANDUTV_OK;
    {
        std::lock_guard<std::mutex> lk(enqueue_lock(dev));
        const cudaError_t e = fo.qr_first ? run_qr_first(c, A, lda, stop_after) : run_factor(c, A, lda, stop_after);
        if (e != cudaSuccess) return RANDUTV_ECUDA;
    }
    if (fo.cols_done) *fo.cols_done = c.cols_done;
    if (fo.rank) *fo.rank = c.rank_tol > 0.0 ? c.rank : c.cols_done;
    if (ma.tr_count) *ma.tr_count = c.tr_count;
    if (info != nullptr) {
        if (cudaMemcpyAsync(info, c.w.status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RANDUTV_ECUDA;
        return RANDUTV_OK;
    }
    if (ma.mode == MODE_LEARNED && ma.q_used && nblocks > 0 &&
        cudaMemcpyAsync(ma.q_used, c.w.qlog, sizeof(int) * (size_t)nblocks, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return RANDUTV_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, c.w.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return RANDUTV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RANDUTV_ECUDA;
    return status_from_bits(bits);
}

}  // namespace
}  // namespace rutv

extern "C" {

randutv_status randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed,
                                 double* U, double* T, double* V, int prec, void* stream, void* workspace,
                                 size_t ws_bytes, int64_t stop_after, int* info) {
    return factor_impl(m, n, A, lda, b, q, seed, U, T, V, prec, stream, workspace, ws_bytes, stop_after, info,
                       ModeArgs{});
}

void randutv_options_init(randutv_options* opt) {
    if (!opt) return;
    *opt = randutv_options{};
    opt->prec = RANDUTV_FP64;
    opt->stop_after = -1;
}

size_t randutv_workspace_size_opt(int64_t m, int64_t n, int b, const randutv_options* opt) {
    if (m < n || n < 0 || b < 1) return 0;
    const int prec = opt ? opt->prec : RANDUTV_FP64;
    if (!valid_prec(prec)) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    return make_layout(m, n, b, device_sms(dev), prec, opt && opt->qr_first).total;
}

randutv_status randutv_factor_opt(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed,
                                  double* U, double* T, double* V, randutv_options* opt) {
    randutv_options o;
    randutv_options_init(&o);
    if (opt) o = *opt;
    if (!(o.rank_tol >= 0.0) || !std::isfinite(o.rank_tol) || o.start_col < 0 || o.start_col > n) return RANDUTV_EINVAL;
    if (o.start_col > 0 && (b < 1 || (o.start_col % b != 0 && o.start_col != n))) return RANDUTV_EINVAL;
    if (o.start_col > 0 && o.qr_first) return RANDUTV_EINVAL;
    FactorOpts fo;
    fo.start_col = o.start_col;
    fo.rank_tol = o.rank_tol;
    fo.qr_first = o.qr_first != 0;
    fo.cols_done = opt ? &opt->cols_done : nullptr;
    fo.rank = opt ? &opt->rank : nullptr;
    // a resumed call does not read A: T stands in for it in the argument checks
    const double* a = (o.start_col > 0) ? T : A;
    const int64_t la = (o.start_col > 0) ? std::max<int64_t>(m, 1) : lda;
    return factor_impl(m, n, a, la, b, q, seed, U, T, V, o.prec, o.stream, o.workspace, o.ws_bytes, o.stop_after,
                       nullptr, ModeArgs{}, fo);
}

randutv_status randutv_factor_learnedq_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b,
                                          const float* model, uint64_t seed, double* U, double* T, double* V,
                                          int* q_used, int prec, void* stream) {
    ModeArgs ma;
    ma.mode = MODE_LEARNED;
    ma.model = model;
    ma.q_used = q_used;
    return factor_impl(m, n, A, lda, b, 2, seed, U, T, V, prec, stream, nullptr, 0, -1, nullptr, ma);
}

randutv_status randutv_factor_learnedq(int64_t m, int64_t n, const double* A, int64_t lda, int b, const float* model,
                                       uint64_t seed, double* U, double* T, double* V, int* q_used) {
    return randutv_factor_learnedq_ex(m, n, A, lda, b, model, seed, U, T, V, q_used, RANDUTV_FP64, nullptr);
}

randutv_status randutv_learnq_trace_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                                       double* T, float* features, int* labels, double* candidates,
                                       int64_t max_blocks, int64_t* nblocks, int prec, int64_t stride) {
    if (!features || !labels || max_blocks < 0 || b > 512 || stride < 1) return RANDUTV_EINVAL;
    if (prec != RANDUTV_FP64 && prec != RANDUTV_FP64_EMULATED) return RANDUTV_EINVAL;
    ModeArgs ma;
    ma.mode = MODE_TRACE;
    ma.tr_feat = features;
    ma.tr_label = labels;
    ma.tr_cand = candidates;
    ma.tr_max = max_blocks;
    ma.tr_stride = stride;
    int64_t cnt = 0;
    ma.tr_count = &cnt;
    randutv_status r =
        factor_impl(m, n, A, lda, b, 2, seed, nullptr, T, nullptr, prec, nullptr, nullptr, 0, -1, nullptr, ma);
    if (nblocks) *nblocks = cnt;
    return r;
}

randutv_status randutv_learnq_trace(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                                    double* T, float* features, int* labels, double* candidates, int64_t max_blocks,
                                    int64_t* nblocks) {
    return randutv_learnq_trace_ex(m, n, A, lda, b, seed, T, features, labels, candidates, max_blocks, nblocks,
                                   RANDUTV_FP64, 1);
}

int randutv_learnq_model_floats(void) { return learnq_nparam(); }

namespace {
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};
}  // namespace

randutv_status randutv_learnq_train(const float* X, const int* y, int N, int epochs, float lr, float wd,
                                    float* model, float* loss_history) {
    if (!X || !y || !model || N <= 0 || epochs < 0) return RANDUTV_EINVAL;
    const int np = learnq_nparam();
    const size_t scr = learnq_train_scratch_floats(N);
    DevBuf buf;
    size_t bytes = sizeof(float) * ((size_t)N * 16 + np + scr + (size_t)std::max(epochs, 1)) + sizeof(int) * N + 1024;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) return RANDUTV_ENOMEM;
    float* dX = (float*)buf.p;
    float* dP = dX + (size_t)N * 16;
    float* dS = dP + np;
    float* dL = dS + scr;
    int* dy = (int*)(dL + std::max(epochs, 1));
    if (cudaMemcpy(dX, X, sizeof(float) * N * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dy, y, sizeof(int) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dP, model, sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dS, 0, sizeof(float) * scr) != cudaSuccess)
        return RANDUTV_ECUDA;
    for (int e = 0; e < epochs; ++e)
        if (learnq_train_step(dP, dX, dy, N, dS, nullptr, dL + e, e + 1, lr, wd, nullptr) != cudaSuccess)
            return RANDUTV_ECUDA;
    if (cudaMemcpy(model, dP, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess) return RANDUTV_ECUDA;
    if (loss_history && epochs > 0 &&
        cudaMemcpy(loss_history, dL, sizeof(float) * epochs, cudaMemcpyDeviceToHost) != cudaSuccess)
        return RANDUTV_ECUDA;
    return RANDUTV_OK;
}

randutv_status randutv_learnq_grad(const float* X, const int* y, int N, const float* model, float* grad,
                                   float* loss) {
    if (!X || !y || !model || !grad || N <= 0) return RANDUTV_EINVAL;
    const int np = learnq_nparam();
    const size_t scr = learnq_train_scratch_floats(N);
    DevBuf buf;
    size_t bytes = sizeof(float) * ((size_t)N * 16 + 2 * (size_t)np + scr + 4) + sizeof(int) * N + 1024;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) return RANDUTV_ENOMEM;
    float* dX = (float*)buf.p;
    float* dP = dX + (size_t)N * 16;
    float* dG = dP + np;
    float* dS = dG + np;
    float* dL = dS + scr;
    int* dy = (int*)(dL + 4);
    if (cudaMemcpy(dX, X, sizeof(float) * N * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dy, y, sizeof(int) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dP, model, sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(dG, 0, sizeof(float) * np) != cudaSuccess)
        return RANDUTV_ECUDA;
    if (learnq_train_step(dP, dX, dy, N, dS, dG, dL, 0, 0.f, 0.f, nullptr) != cudaSuccess) return RANDUTV_ECUDA;
    if (cudaMemcpy(grad, dG, sizeof(float) * np, cudaMemcpyDeviceToHost) != cudaSuccess) return RANDUTV_ECUDA;
    if (loss && cudaMemcpy(loss, dL, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return RANDUTV_ECUDA;
    return RANDUTV_OK;
}

randutv_status randutv_learnq_predict(const float* model, const float* X, int N, float* probs) {
    if (!model || !X || !probs || N <= 0) return RANDUTV_EINVAL;
    const int np = learnq_nparam();
    DevBuf buf;
    if (cudaMalloc(&buf.p, sizeof(float) * ((size_t)N * 20 + np) + 256) != cudaSuccess) return RANDUTV_ENOMEM;
    float* dX = (float*)buf.p;
    float* dP = dX + (size_t)N * 16;
    float* dPr = dP + np;
    if (cudaMemcpy(dX, X, sizeof(float) * N * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dP, model, sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess)
        return RANDUTV_ECUDA;
    if (learnq_predict(dP, dX, N, dPr, nullptr) != cudaSuccess) return RANDUTV_ECUDA;
    if (cudaMemcpy(probs, dPr, sizeof(float) * N * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return RANDUTV_ECUDA;
    return RANDUTV_OK;
}

randutv_status randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q, uint64_t seed,
                              double* U, double* T, double* V) {
    return randutv_factor_ex(m, n, A, lda, b, q, seed, U, T, V, RANDUTV_FP64, nullptr, nullptr, 0, -1, nullptr);
}

randutv_status randutv_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                                   uint64_t seed, double* U, double* T, double* V, int prec) {
    if (!args_ok(m, n, A, lda, b, q, T)) return RANDUTV_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RANDUTV_ECUDA;
    const size_t bytesT = sizeof(double) * (size_t)m * n;
    const size_t bytesU = sizeof(double) * (size_t)m * m, bytesV = sizeof(double) * (size_t)n * n;
    void *dA = nullptr, *dU = nullptr, *dV = nullptr;
    if (cached_buffer(dev, 0, std::max<size_t>(bytesT, 8), &dA) != cudaSuccess) return RANDUTV_ENOMEM;
    if (U && cached_buffer(dev, 1, std::max<size_t>(bytesU, 8), &dU) != cudaSuccess) return RANDUTV_ENOMEM;
    if (V && cached_buffer(dev, 2, std::max<size_t>(bytesV, 8), &dV) != cudaSuccess) return RANDUTV_ENOMEM;
    cudaStream_t st = nullptr;  // legacy default stream
    const int sms = device_sms(dev);
    if (bytesT > 0) {
        // pinned host memory: the SMs copy from it directly; otherwise one
        // contiguous DMA copy when A has no padding, else a pitched one
        const double* hA = (const double*)pinned_device_address(A);
        cudaError_t e;
        if (hA && lda == m)
            e = copy_flat(hA, (double*)dA, m * n, sms, st);
        else if (hA)
            e = copy_matrix(hA, lda, (double*)dA, m, m, n, st);
        else
            e = (lda == m) ? cudaMemcpyAsync(dA, A, bytesT, cudaMemcpyHostToDevice, st)
                           : cudaMemcpy2DAsync(dA, sizeof(double) * m, A, sizeof(double) * lda, sizeof(double) * m,
                                               n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return RANDUTV_ECUDA;
    }
    randutv_status rs = randutv_factor_ex(m, n, (double*)dA, m, b, q, seed, (double*)dU, (double*)dA, (double*)dV,
                                          prec, st, nullptr, 0, -1, nullptr);
    if ((rs == RANDUTV_OK || rs == RANDUTV_ENOCONV) && bytesT > 0) {
        auto out = [&](double* host, const void* src, size_t bytes) -> cudaError_t {
            double* h = (double*)pinned_device_address(host);
            return h ? copy_flat((const double*)src, h, (int64_t)(bytes / sizeof(double)), sms, st)
                     : cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, st);
        };
        if (out(T, dA, bytesT) != cudaSuccess) return RANDUTV_ECUDA;
        if (U && out(U, dU, bytesU) != cudaSuccess) return RANDUTV_ECUDA;
        if (V && out(V, dV, bytesV) != cudaSuccess) return RANDUTV_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return RANDUTV_ECUDA;
    }
    return rs;
}

}  // extern "C"
