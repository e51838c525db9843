// ff_host.cuh -- host-side helpers shared by the library's translation units:
// argument checks, CUDA error capture, device properties and launch sizing.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ff.h"

namespace ffh {

// Remember a CUDA error for ff_last_cuda_error() (thread-local).
void set_cuda_error(cudaError_t e);

// FF_OK if no launch error is pending, else FF_ERR_CUDA (error recorded).
inline ff_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return FF_ERR_CUDA;
    }
    return FF_OK;
}

inline ff_status cuda_status(cudaError_t e)
{
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return FF_ERR_CUDA;
    }
    return FF_OK;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// A device array argument: non-NULL when it holds elements, 8-byte aligned.
inline bool ok_ptr(const void* p, size_t n) { return n == 0 || (p != nullptr && aligned(p, 8)); }

struct DeviceInfo {
    int device;
    int sm_count;
    int max_threads_per_sm;
};

// Properties of the current device (cached per device).
ff_status device_info(DeviceInfo* out);

// Blocks per SM for `kernel` launched with `block` threads (cached by the
// caller in a function-local static keyed by device when needed).
int occupancy(const void* kernel, int block, size_t smem = 0);

// Grid for a grid-stride kernel: enough blocks to cover `work` items of
// `per_block` each, capped at SMs x resident blocks per SM.
inline unsigned grid_for(size_t work, size_t per_block, int sm_count, int blocks_per_sm)
{
    size_t want = (work + per_block - 1) / per_block;
    size_t cap = static_cast<size_t>(sm_count) * static_cast<size_t>(blocks_per_sm > 0 ? blocks_per_sm : 1);
    if (want < 1) want = 1;
    return static_cast<unsigned>(want < cap ? want : cap);
}

}  // namespace ffh
