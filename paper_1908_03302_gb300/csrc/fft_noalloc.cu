// One point-spread function without any device allocation.
//
// fft_psf_batch allocates its per-call scratch (the column J_S e_k and a copy of the row
// lists) with cudaMalloc. Some callers cannot allow that: code that must not touch the
// allocator once it is running (a service that reserves all device memory at start-up,
// or a memory pool owned by another framework whose budget a stray cudaMalloc would break),
// and code that must not block the device, since cudaMalloc / cudaFree may synchronise.
// fft_psf_noalloc computes the same quantity for one spike and one row subset with its
// scratch in a file-scope device array of fixed size instead.
//
// The array (NOALLOC_MAX_ROWS floats plus a 256-byte header, about 16 MB) belongs to this
// file's device module. With CUDA's lazy module loading that module, and the 16 MB, are
// committed on a device the first time anything in it is used; fft_geom_create does that
// (noalloc_prepare below), so the device memory is taken when the first geometry is created
// on a device and held until the process exits, and fft_psf_noalloc itself loads and
// allocates nothing. All calls share the array and it keeps the last call's contents; each
// call clears the part it uses first. Calls that overlap on the GPU (different streams, or
// several host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "fft_common.cuh"
#include "fft_device.cuh"

namespace fftgb {

namespace {

constexpr int64_t NOALLOC_MAX_ROWS = int64_t(1) << 22;   // 4,194,304 rows
constexpr int NOALLOC_HEADER_FLOATS = 64;                // 256 bytes: error counter + padding
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_HEADER_FLOATS + NOALLOC_MAX_ROWS];

std::mutex g_setup_mutex;
float* g_scratch_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device,
// with that device current; the host-side symbol is only a stand-in, never a device pointer).
fft_status scratch_for_device(int dev, float** out) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("fft_psf_noalloc: device index out of range");
        return FFT_ERR_STATE;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "fft_psf_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return FFT_OK;
}

// D[rows[i]] = J[rows[i], v]; row indices outside [0, M) are counted in *err and skipped.
template <int DT>
__global__ void noalloc_column_kernel(const RowRec* __restrict__ rec, const int32_t* __restrict__ row_band,
                                      const BandConst* __restrict__ bc, const float2* __restrict__ tab, int n_tab,
                                      const int32_t* __restrict__ rows, int n, int64_t M, int nx, int ny,
                                      int64_t v, const RowRec64* __restrict__ rec64, double3 org64, double h64,
                                      float* __restrict__ D, unsigned int* __restrict__ err);

}  // namespace

// Look the array's device address up with `dev` current (the host-side symbol is only a
// stand-in) and load the column kernels, so the first fft_psf_noalloc call on the device has
// nothing left to load.
fft_status noalloc_prepare(int dev) {
    float* p = nullptr;
    fft_status rc = scratch_for_device(dev, &p);
    if (rc != FFT_OK) return rc;
    cudaFuncAttributes fa;
    FFT_CUDA(cudaFuncGetAttributes(&fa, noalloc_column_kernel<FFT_DT_STABLE>));
    FFT_CUDA(cudaFuncGetAttributes(&fa, noalloc_column_kernel<FFT_DT_NAIVE>));
    return FFT_OK;
}

namespace {

template <int DT>
__global__ void noalloc_column_kernel(const RowRec* __restrict__ rec, const int32_t* __restrict__ row_band,
                                      const BandConst* __restrict__ bc, const float2* __restrict__ tab, int n_tab,
                                      const int32_t* __restrict__ rows, int n, int64_t M, int nx, int ny,
                                      int64_t v, const RowRec64* __restrict__ rec64, double3 org64, double h64,
                                      float* __restrict__ D, unsigned int* __restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = rows[i];
    if (p < 0 || p >= M) {
        atomicAdd(err, 1u);
        return;
    }
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
    D[p] = phi_lookup_global(vv, tab + (int64_t)b * n_tab, n_tab) * (is * ir) * r.b.w;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_psf_noalloc(fft_geom g, int64_t spike_vox, const int32_t* rows_dev, int32_t n_rows,
                                      float* out_dev, void* stream) {
    FFT_ARG(g && out_dev, "fft_psf_noalloc: null argument");
    FFT_ARG(n_rows >= 0 && (n_rows == 0 || rows_dev), "fft_psf_noalloc: need n_rows >= 0 and rows_dev");
    FFT_ARG(spike_vox >= 0 && spike_vox < g->V, "fft_psf_noalloc: spike voxel out of range");
    FFT_ARG(g->phi_kind == PHI_TABLE, "fft_psf_noalloc: needs a geometry built from sampled tables (not sine series)");
    if (g->M > NOALLOC_MAX_ROWS) {
        set_error("fft_psf_noalloc: the geometry has more rows than the static scratch holds (4194304)");
        return FFT_ERR_ARG;
    }
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    float* base = nullptr;
    if ((rc = scratch_for_device(g->dev, &base)) != FFT_OK) return rc;
    unsigned int* err = reinterpret_cast<unsigned int*>(base);
    float* D = base + NOALLOC_HEADER_FLOATS;
    cudaStream_t st = (cudaStream_t)stream;

    // the error counter and the column must start at zero; the previous call left its values
    FFT_CUDA(cudaMemsetAsync(base, 0, sizeof(float) * (NOALLOC_HEADER_FLOATS + g->M), st));
    if (n_rows > 0) {
        const unsigned blocks = (unsigned)ceil_div(n_rows, 256);
        if (g->dt_mode == FFT_DT_NAIVE)
            noalloc_column_kernel<FFT_DT_NAIVE><<<blocks, 256, 0, st>>>(
                g->rec, g->row_band, g->d_band, g->tab, g->n_tab, rows_dev, n_rows, g->M, g->grid.nx, g->grid.ny,
                spike_vox, g->rec64, make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]), g->grid.h,
                D, err);
        else
            noalloc_column_kernel<FFT_DT_STABLE><<<blocks, 256, 0, st>>>(
                g->rec, g->row_band, g->d_band, g->tab, g->n_tab, rows_dev, n_rows, g->M, g->grid.nx, g->grid.ny,
                spike_vox, g->rec64, make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]), g->grid.h,
                D, err);
        FFT_CUDA(cudaGetLastError());
    }
    if ((rc = launch_JT(g, D, out_dev, st)) != FFT_OK) return rc;
    unsigned int bad = 0;
    FFT_CUDA(cudaMemcpyAsync(&bad, err, sizeof(bad), cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaStreamSynchronize(st));
    if (bad) {
        set_error("fft_psf_noalloc: " + std::to_string(bad) + " row indices were outside [0, M) (M = " +
                  std::to_string(g->M) + ", the geometry's row count) and skipped");
        return FFT_ERR_ARG;
    }
    return FFT_OK;
}
