// Error reporting and small helpers shared by the C ABI entry points.
#include <cuda_runtime.h>

#include <string>

#include "fft_common.cuh"

namespace fftgb {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

fft_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return FFT_ERR_OOM;
    return FFT_ERR_CUDA;
}

// Calls on a handle must run with the handle's device current.
fft_status check_device(int dev) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != dev) {
        set_error("handle belongs to device " + std::to_string(dev) + " but device " + std::to_string(cur) +
                  " is current");
        return FFT_ERR_STATE;
    }
    return FFT_OK;
}

}  // namespace fftgb

extern "C" const char* fft_last_error(void) { return fftgb::g_last_error.c_str(); }
