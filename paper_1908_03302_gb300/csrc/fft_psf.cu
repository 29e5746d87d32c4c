// Hessian point-spread functions H_S e_k = J_S^T J_S e_k (Sec. II-D, Eq. resolution_2): the
// misfit Hessian applied to a unit perturbation at voxel k, restricted to a subset S of rows
// (a ring subset of the acquisition).
//
// FP32 CUDA-core path: column k of J_S is evaluated row by row (one thread per row of S),
// then J^T is applied to it. J^T skips rows whose weight is zero, so the cost of each PSF
// follows the rows whose support holds the spike.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "fft_common.cuh"
#include "fft_device.cuh"

namespace fftgb {

namespace {

// D[rows[i]] = J[rows[i], v] for i < n (voxel v), evaluated like the apply kernels: pair
// frame in band units, cancellation-free detour, linear interpolation of the band table.
template <int DT>
__global__ void column_kernel(const RowRec* __restrict__ rec, const int32_t* __restrict__ row_band,
                              const BandConst* __restrict__ bc, const float2* __restrict__ tab, int n_tab,
                              const int32_t* __restrict__ rows, int n, int nx, int ny, int64_t v,
                              const RowRec64* __restrict__ rec64, double3 org64, double h64,
                              float* __restrict__ D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = rows[i];
    const RowRec r = rec[p];
    const int b = row_band[p];
    const BandConst c = bc[b];
    const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((int64_t)nx * ny));
    const float dx = fmaf((float)ix, c.h, c.org[0]) - r.a.x;
    const float dy = fmaf((float)iy, c.h, c.org[1]) - r.a.y;
    const float dz = fmaf((float)iz, c.h, c.org[2]) - r.a.z;
    const float ex = r.b.x, ey = r.b.y, ez = r.b.z;
    const float pp = fmaf(dx, ex, fmaf(dy, ey, dz * ez));
    const float c1 = fmaf(dy, ez, -dz * ey), c2 = fmaf(dz, ex, -dx * ez), c3 = fmaf(dx, ey, -dy * ex);
    const float q2 = fmaf(c1, c1, fmaf(c2, c2, c3 * c3));
    float is, ir;
    float vv = detour_v<DT == FFT_DT_NAIVE ? FFT_DT_NAIVE : FFT_DT_STABLE, true, false, true>(pp + r.a.w, pp - r.a.w,
                                                                                            q2, r.a.w, is, ir);
    if (c.sharp && fabsf(vv - 1.0f) < CUT_BAND)   // decide the cut of a sharp band in FP64
        vv = settle_cut(__saturatef(vv), in_support64(rec64[p], org64.x, org64.y, org64.z, h64, ix, iy, iz, c.U));
    vv = __saturatef(vv);
    const float nm1 = (float)(n_tab - 1);
    const float u = vv * nm1;
    int k = (int)floorf(u);
    if (k > n_tab - 1) k = n_tab - 1;
    if (k < 0) k = 0;
    const float2 T = tab[(int64_t)b * n_tab + k];
    const float phi = fmaf(u - (float)k, T.y, T.x);
    D[p] = phi * (is * ir) * r.b.w;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_psf_batch(fft_geom g, const int64_t* spike_vox, int32_t n_spike,
                                    const int32_t* subset_off, int32_t n_subsets, const int32_t* subset_rows,
                                    int32_t mode, float* out_dev, void* stream) {
    FFT_ARG(g && spike_vox && subset_off && out_dev, "fft_psf_batch: null argument");
    FFT_ARG(n_spike >= 1 && n_subsets >= 1, "fft_psf_batch: need at least one spike and one subset");
    FFT_ARG(mode == 0, "fft_psf_batch: mode must be 0 (FP32)");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    for (int k = 0; k < n_spike; ++k)
        FFT_ARG(spike_vox[k] >= 0 && spike_vox[k] < g->V, "fft_psf_batch: spike voxel out of range");
    FFT_ARG(subset_off[0] == 0, "fft_psf_batch: subset_off[0] must be 0");
    for (int s = 0; s < n_subsets; ++s)
        FFT_ARG(subset_off[s + 1] >= subset_off[s], "fft_psf_batch: subset offsets must be non-decreasing");
    const int32_t n_idx = subset_off[n_subsets];
    FFT_ARG(n_idx == 0 || subset_rows, "fft_psf_batch: null subset_rows");
    for (int32_t i = 0; i < n_idx; ++i)
        FFT_ARG(subset_rows[i] >= 0 && subset_rows[i] < g->M, "fft_psf_batch: subset row out of range");

    cudaStream_t st = (cudaStream_t)stream;
    int32_t* d_rows = nullptr;
    float* D = nullptr;
    FFT_CUDA(cudaMalloc(&d_rows, sizeof(int32_t) * (n_idx > 0 ? n_idx : 1)));
    cudaError_t e = cudaMalloc(&D, sizeof(float) * g->M);
    if (e != cudaSuccess) {
        cudaFree(d_rows);
        return cuda_fail(e, "fft_psf_batch cudaMalloc");
    }
    if (n_idx > 0) e = cudaMemcpyAsync(d_rows, subset_rows, sizeof(int32_t) * n_idx, cudaMemcpyHostToDevice, st);
    for (int s = 0; s < n_subsets && e == cudaSuccess && rc == FFT_OK; ++s) {
        const int32_t a = subset_off[s], n = subset_off[s + 1] - a;
        for (int k = 0; k < n_spike && e == cudaSuccess && rc == FFT_OK; ++k) {
            e = cudaMemsetAsync(D, 0, sizeof(float) * g->M, st);
            if (e != cudaSuccess) break;
            if (n > 0) {
                if (g->dt_mode == FFT_DT_NAIVE)
                    column_kernel<FFT_DT_NAIVE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                        g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                        spike_vox[k], g->rec64, make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]),
                        g->grid.h, D);
                else
                    column_kernel<FFT_DT_STABLE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                        g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                        spike_vox[k], g->rec64, make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]),
                        g->grid.h, D);
                e = cudaGetLastError();
                if (e != cudaSuccess) break;
            }
            rc = launch_JT(g, D, out_dev + ((int64_t)s * n_spike + k) * g->V, st);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(d_rows);
    cudaFree(D);
    if (rc != FFT_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fft_psf_batch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "fft_psf_batch sync");
    return FFT_OK;
}
