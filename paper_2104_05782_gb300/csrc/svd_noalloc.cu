// svd_noalloc.cu -- an allocation-free entry point for the b x b SVD step.
//
// Some callers cannot allocate device memory at all: code running under a
// memory pool or arena that forbids cudaMalloc, allocation-free real-time
// paths, or plugins whose host framework owns every allocation.  For them the
// one-sided Jacobi SVD of the diagonal block (the kernel randutv_factor runs
// for every block step) is offered with its scratch in a file-scope device
// array instead of a workspace: the Jacobi working copies of A and V, the
// grid-barrier counter, the rotation counters and the status word.  The array
// is sized for w <= RANDUTV_SVD_NOALLOC_MAX_W and every GPU that loads the
// library keeps it (about 1 MiB) until the process exits.
#include <mutex>

#include "../../include/randutv.h"
#include "common.cuh"
#include "internal.h"

namespace rutv {

namespace {

constexpr int kMaxW = RANDUTV_SVD_NOALLOC_MAX_W;
constexpr size_t kWork = (size_t)2 * kMaxW * kMaxW;  // Jacobi copies of A and V
constexpr size_t kTail = 16;                          // barrier, 3 rotation counters, status (as doubles)
constexpr int kMaxDevices = 64;

// Shared by every call on a device; see the entry point's notes on overlap.
static __device__ __align__(256) double g_svd_scratch[kWork + kTail];

// Device address of g_svd_scratch, looked up once per device (under a lock,
// so that host threads calling for the first time do not race).  A host-side
// reference to the symbol is only a stand-in, never a device address.
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Looks up the device address of the scratch array on the current device.
bool scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_svd_scratch) != cudaSuccess || p == nullptr) return false;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return true;
}

}  // namespace

}  // namespace rutv

using namespace rutv;

extern "C" randutv_status randutv_svd_small_noalloc(int w, const double* R, int64_t ldr, double* D, double* Us,
                                                    double* Vs, void* stream) {
    if (w < 0 || w > kMaxW) return RANDUTV_EINVAL;
    if (w == 0) return RANDUTV_OK;
    if (!R || !D || !Us || !Vs || ldr < w) return RANDUTV_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RANDUTV_ECUDA;
    void* addr = nullptr;
    if (!scratch_address(dev, &addr)) return RANDUTV_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    double* base = (double*)addr;
    unsigned* bar = (unsigned*)(base + kWork);
    int* counters = (int*)(base + kWork + 2);
    int* status = (int*)(base + kWork + 4);
    // the barrier counter is zeroed by the launcher, the rotation counters by
    // the kernel itself; the status word is cleared here
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return RANDUTV_ECUDA;
    if (jacobi_svd(R, ldr, w, D, Us, Vs, base, bar, counters, status, sweep_cap(), st, /*allow_cluster=*/false) != cudaSuccess)
        return RANDUTV_ECUDA;
    int bits = 0;
    if (cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RANDUTV_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RANDUTV_ECUDA;
    if (bits & ST_TIMEOUT) return RANDUTV_ETIMEOUT;
    if (bits & ST_NONFINITE) return RANDUTV_ENONFINITE;
    if (bits & ST_NOCONV) return RANDUTV_ENOCONV;
    return RANDUTV_OK;
}
