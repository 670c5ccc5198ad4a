// Device and pinned host allocations of the create calls (rule sets, learned
// indexes, plans, servers, host pipelines) go through these two wrappers, so
// that a test hook (fw_selftest_fail_alloc) can make one of them fail as if
// memory ran out, on the host, without a GPU fault.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace fwk {

// True exactly once, at the allocation the hook armed (then the hook disarms).
bool take_injected_alloc_failure();

template <class T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    if (take_injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

template <class T>
cudaError_t pinned_malloc(T **p, size_t bytes) {
    if (take_injected_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}

}  // namespace fwk
