// Device allocations of the library go through these two calls (all but the
// 4-byte status word of pm_selftest_bounded_wait), so that a test can make
// one of them fail on the host (pm_debug_fail_alloc in pm.h) and check that
// the failure comes back as PM_ERR_OOM with nothing launched on the memory
// that was never obtained.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

// Device memory from the library's pool of the current device, ready for any
// stream when the call returns (as cudaMalloc's); or cudaErrorMemoryAllocation
// without calling CUDA when the armed failure is due.
cudaError_t pm_device_malloc(void **ptr, size_t bytes);

// Releases memory of pm_device_malloc after every launch on its device has
// finished (as cudaFree waits); the pool keeps it for later allocations.
void pm_device_free(void *ptr);

// Stream-ordered memory from the same pool on stream s (released with
// cudaFreeAsync on s), with the same injected failure.
cudaError_t pm_device_malloc_async(void **ptr, size_t bytes, cudaStream_t s);
