// Device allocations of the library go through these two calls (all but the
// 4-byte status word of pm_selftest_bounded_wait), so that a test can make
// one of them fail on the host (pm_debug_fail_alloc in pm.h) and check that
// the failure comes back as PM_ERR_OOM with nothing launched on the memory
// that was never obtained.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

// cudaMalloc, or cudaErrorMemoryAllocation without calling CUDA when the
// armed failure is due.
cudaError_t pm_device_malloc(void **ptr, size_t bytes);

// cudaMallocAsync on stream s, with the same injected failure.
cudaError_t pm_device_malloc_async(void **ptr, size_t bytes, cudaStream_t s);
