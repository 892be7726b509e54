// trace.h -- per-kernel-class CUDA-event tracing and launch counting.
//
// The paper studies where the time of a randUTV step goes (Sec. 5.4; execution
// traces of Sec. 6.1).  Here every launcher of the library runs inside a
// TraceScope: when tracing is on, a pair of CUDA events brackets the launch
// on its own stream and the algorithmic flops / bytes of that launch are
// recorded under a class name; the library-wide kernel-launch counter is
// always maintained.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rutv {

struct TraceScope {
    TraceScope(const char* cls, double flops, double bytes, cudaStream_t st);
    ~TraceScope();
    const char* cls_;
    double flops_, bytes_;
    cudaStream_t st_;
    int slot_;
    long long start_;
};

void trace_count(int kernels);

}  // namespace rutv
