// Self-test of the tcgen05 building blocks (fft_tc.cuh): one 128 x N x K BF16 product with
// integer-valued operands, whose FP32 result is exact, so any layout or descriptor mistake
// shows up as a non-zero difference.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "fft_common.cuh"
#include "fft_device.cuh"
#include "fft_tc.cuh"

namespace fftgb {

namespace {

constexpr int ST_THREADS = 128;

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, long long budget_cycles) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(mbar, parity)) {
        if (clock64() - t0 > budget_cycles) return false;
    }
    return true;
}

// A: 128 x K row-major BF16 (global), B: N x K row-major BF16, C: 128 x N FP32.
__global__ void __launch_bounds__(ST_THREADS) tc_selftest_kernel(const __nv_bfloat16* __restrict__ A,
                                                                 const __nv_bfloat16* __restrict__ B, int N,
                                                                 int K, float* __restrict__ C,
                                                                 int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = 128u * (uint32_t)K * 2u;
    unsigned char* sA = smem;
    unsigned char* sB = smem + a_bytes;

    for (int i = tid; i < 128 * K; i += ST_THREADS) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__nv_bfloat16*>(sA + tc::kmajor_offset(r, k, K)) = A[i];
    }
    for (int i = tid; i < N * K; i += ST_THREADS) {
        const int r = i / K, k = i % K;
        *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(r, k, K)) = B[i];
    }
    const uint32_t mbar_addr = smem_addr(&mbar);
    if (warp == 0) {
        tc::tmem_alloc(smem_addr(&tmem_slot), (uint32_t)N);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(mbar_addr, 1);
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_slot;

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)N);
        const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(a0 + 256u * ks, 128u, 16u * (uint32_t)K);
            const uint64_t bd = tc::smem_desc(b0 + 256u * ks, 128u, 16u * (uint32_t)K);
            tc::mma_bf16(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(mbar_addr);
    }
    // bounded wait (~1 s at 2 GHz); on time-out record it, wait once more, then clean up
    bool ok = wait_phase(mbar_addr, 0, 2000000000ll);
    if (!ok) {
        if (lane == 0) atomicExch(status, FFT_ERR_TIMEOUT);
        ok = wait_phase(mbar_addr, 0, 2000000000ll);
    }
    tc::fence_after_sync();
    if (ok) {
        const uint32_t row = 32u * (uint32_t)warp + (uint32_t)lane;
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc::tmem_ld_x8(taddr + ((32u * (uint32_t)warp) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) C[(size_t)row * N + c + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)N);
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_tc_selftest(int32_t n, int32_t k, double* max_abs_err) {
    FFT_ARG(max_abs_err, "fft_tc_selftest: null output");
    FFT_ARG(n == 32 || n == 64 || n == 128 || n == 256, "fft_tc_selftest: n must be 32, 64, 128 or 256");
    FFT_ARG(k >= 16 && k <= 256 && k % 16 == 0, "fft_tc_selftest: k must be a multiple of 16 in [16, 256]");
    const int M = 128;
    std::vector<__nv_bfloat16> a((size_t)M * k), b((size_t)n * k);
    std::vector<float> af((size_t)M * k), bf((size_t)n * k);
    for (int r = 0; r < M; ++r)
        for (int j = 0; j < k; ++j) {
            float v = (float)((r * 5 + j * 3) % 13 - 6);
            af[(size_t)r * k + j] = v;
            a[(size_t)r * k + j] = __float2bfloat16(v);
        }
    for (int r = 0; r < n; ++r)
        for (int j = 0; j < k; ++j) {
            float v = (float)((r * 7 + j * 11) % 11 - 5);
            bf[(size_t)r * k + j] = v;
            b[(size_t)r * k + j] = __float2bfloat16(v);
        }
    __nv_bfloat16 *dA = nullptr, *dB = nullptr;
    float* dC = nullptr;
    int* dS = nullptr;
    fft_status rc = FFT_OK;
    cudaError_t e = cudaMalloc(&dA, a.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dB, b.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dC, sizeof(float) * M * n);
    if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, a.data(), a.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, b.data(), b.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dC, 0xFF, sizeof(float) * M * n);   // NaN pattern
    if (e == cudaSuccess) e = cudaMemset(dS, 0, sizeof(int));
    const size_t smem = (size_t)(M + n) * k * 2;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        tc_selftest_kernel<<<1, ST_THREADS, smem>>>(dA, dB, n, k, dC, dS);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<float> c((size_t)M * n);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(c.data(), dC, sizeof(float) * M * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, dS, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dS);
    if (e != cudaSuccess) return cuda_fail(e, "fft_tc_selftest");
    if (st != 0) {
        set_error("fft_tc_selftest: the MMA completion wait timed out");
        return FFT_ERR_TIMEOUT;
    }
    double worst = 0.0;
    for (int r = 0; r < M; ++r)
        for (int j = 0; j < n; ++j) {
            double ref = 0.0;
            for (int q = 0; q < k; ++q) ref += (double)af[(size_t)r * k + q] * (double)bf[(size_t)j * k + q];
            double d = fabs((double)c[(size_t)r * n + j] - ref);
            if (!(d == d)) d = INFINITY;
            if (d > worst) worst = d;
        }
    *max_abs_err = worst;
    return rc;
}
