// 2-D approximation of the operator (Sec. II-B, Eq. forward_2D): for transducers in one plane
// and a model that varies slowly in z over the kernels' extent, the traveltime is the plane
// integral of the z-integrated kernel times dc(x, y). The z integral is taken by the midpoint
// rule on the geometry's z layers (the same rule as the volume integral, Eq. forward_compact):
//   J2[p, (i, j)] = sum_k J[p, (i, j, k)],   i.e.  J2 = J E  and  J2^T = E^T J^T,
// with E the extrusion of an (nx, ny) map along the nz layers. J2 m2 extrudes m2 into the
// geometry's volume scratch and applies J; J2^T d applies J^T into the scratch and sums each
// column over k in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "fft_common.cuh"

namespace fftgb {

namespace {

__global__ void extrude_kernel(const float* __restrict__ m2, int64_t n2, int nz, float* __restrict__ m3) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n2 * nz) return;
    m3[v] = __ldg(m2 + v % n2);
}

__global__ void zsum_kernel(const float* __restrict__ g3, int64_t n2, int nz, float* __restrict__ g2) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n2) return;
    float s = 0.0f;
    for (int k = 0; k < nz; ++k) s += g3[(int64_t)k * n2 + u];
    g2[u] = s;
}

fft_status vol_scratch(fft_geom g, float** out) {
    if (!g->vol) {
        cudaError_t e = cudaMalloc(&g->vol, sizeof(float) * (size_t)g->V);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("2-D apply: cudaMalloc of the volume scratch failed");
            return FFT_ERR_OOM;
        }
        g->scratch_bytes += (int64_t)(sizeof(float) * (size_t)g->V);
    }
    *out = g->vol;
    return FFT_OK;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_J2d_apply(fft_geom g, const float* m2_dev, float* d_dev, void* stream) {
    FFT_API_RANGE("fft_J2d_apply");
    FFT_ARG(g && m2_dev && d_dev, "fft_J2d_apply: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    float* m3 = nullptr;
    if ((rc = vol_scratch(g, &m3)) != FFT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n2 = (int64_t)g->grid.nx * g->grid.ny;
    extrude_kernel<<<(unsigned)ceil_div(g->V, 256), 256, 0, st>>>(m2_dev, n2, g->grid.nz, m3);
    FFT_CUDA(cudaGetLastError());
    return launch_J(g, m3, d_dev, st);
}

extern "C" fft_status fft_JT2d_apply(fft_geom g, const float* d_dev, float* g2_dev, void* stream) {
    FFT_API_RANGE("fft_JT2d_apply");
    FFT_ARG(g && d_dev && g2_dev, "fft_JT2d_apply: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    float* g3 = nullptr;
    if ((rc = vol_scratch(g, &g3)) != FFT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = launch_JT(g, d_dev, g3, st)) != FFT_OK) return rc;
    const int64_t n2 = (int64_t)g->grid.nx * g->grid.ny;
    zsum_kernel<<<(unsigned)ceil_div(n2, 256), 256, 0, st>>>(g3, n2, g->grid.nz, g2_dev);
    FFT_CUDA(cudaGetLastError());
    return FFT_OK;
}
