// ff_abi.cu -- status strings, CUDA error capture and the cached device
// queries every entry point uses.
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "ff_host.cuh"

#ifndef FF_BUILD_ID
#define FF_BUILD_ID "dev"
#endif

namespace ffh {

static thread_local int g_last_cuda_error = 0;

void set_cuda_error(cudaError_t e) { g_last_cuda_error = static_cast<int>(e); }

ff_status device_info(DeviceInfo* out)
{
    constexpr int kMaxDev = 64;
    static DeviceInfo cache[kMaxDev];
    static bool valid[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDev) return FF_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (valid[dev]) {
            *out = cache[dev];
            return FF_OK;
        }
    }
    DeviceInfo d{};
    d.device = dev;
    e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return cuda_status(e);
    {
        std::lock_guard<std::mutex> lk(mu);
        cache[dev] = d;
        valid[dev] = true;
    }
    *out = d;
    return FF_OK;
}

int occupancy(const void* kernel, int block, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    auto key = std::make_tuple(kernel, block, smem, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int blocks = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, block, smem) != cudaSuccess ||
        blocks < 1) {
        cudaGetLastError();  // clear, fall back to one block per SM
        blocks = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = blocks;
    return blocks;
}

}  // namespace ffh

extern "C" {

const char* ff_status_string(ff_status st)
{
    switch (st) {
    case FF_OK: return "FF_OK";
    case FF_ERR_INVALID_ARG: return "FF_ERR_INVALID_ARG";
    case FF_ERR_WORKSPACE: return "FF_ERR_WORKSPACE";
    case FF_ERR_CUDA: return "FF_ERR_CUDA";
    case FF_ERR_TIMEOUT: return "FF_ERR_TIMEOUT";
    case FF_ERR_UNSUPPORTED: return "FF_ERR_UNSUPPORTED";
    }
    return "FF_ERR_UNKNOWN";
}

ff_status ff_last_cuda_error(int* cuda_err)
{
    if (!cuda_err) return FF_ERR_INVALID_ARG;
    *cuda_err = ffh::g_last_cuda_error;
    return FF_OK;
}

const char* ff_build_id(void) { return FF_BUILD_ID; }

}  // extern "C"
