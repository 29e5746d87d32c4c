// Autotuning of the J / J^T work decomposition. The tile (16 x 16 x 8 voxels) is cut into
// work items of a tile and a range of its candidate rows; how many rows an item takes (set
// through the number of items per persistent CTA) trades load balance at the end of a launch
// against per-item overhead and J^T partial slots, and the persistent grid may hold fewer
// CTAs per SM than fit. Both depend on the acquisition, so they are chosen by timing J and
// J^T on the device for each candidate and keeping the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fft_common.cuh"

namespace fftgb {

namespace {

__global__ void tune_fill_kernel(float* x, int64_t n, float scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = scale * (float)((i * 2654435761u) % 1000u - 500) * 1e-3f;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_geom_autotune(fft_geom g, void* stream, fft_tune_info_t* info) {
    FFT_API_RANGE("fft_geom_autotune");
    FFT_ARG(g, "fft_geom_autotune: null geometry");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    FFT_CUDA(cudaGetDevice(&dev));
    FFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = std::max(1, apply_occupancy(g) / std::max(sms, 1));
    std::vector<int64_t> toff(g->n_tiles + 1);
    FFT_CUDA(cudaMemcpy(toff.data(), g->tile_off, sizeof(int64_t) * (g->n_tiles + 1), cudaMemcpyDeviceToHost));

    float *m = nullptr, *d = nullptr, *out_v = nullptr, *out_m = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    cudaError_t e = cudaMalloc(&m, sizeof(float) * (size_t)g->V);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(float) * (size_t)g->M);
    if (e == cudaSuccess) e = cudaMalloc(&out_v, sizeof(float) * (size_t)g->V);
    if (e == cudaSuccess) e = cudaMalloc(&out_m, sizeof(float) * (size_t)g->M);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&e2);
    if (e == cudaSuccess) {
        tune_fill_kernel<<<(unsigned)ceil_div(g->V, 256), 256, 0, st>>>(m, g->V, 1.0f);
        tune_fill_kernel<<<(unsigned)ceil_div(g->M, 256), 256, 0, st>>>(d, g->M, 1e-8f);
        e = cudaGetLastError();
    }
    // Search: all item sizes at the occupancy limit (stopping once two sizes in a row are
    // slower than the best by more than 2 %), then one CTA per SM fewer around the best size.
    // A candidate gets an untimed pass first unless the last application took over 20 ms
    // (then first-launch effects are lost in the measurement and the pass would double the
    // cost of tuning a large acquisition).
    const int cand_items[] = {4, 8, 16, 32, 64, 128};
    const int n_cand = 6;
    double best = 1e300, best_j = 0.0, best_jt = 0.0, last = 0.0;
    int best_items = g->items_per_cta, best_ctas = g->apply_ctas / std::max(sms, 1), tried = 0, best_ii = 0;
    auto try_one = [&](int ctas, int ii) -> bool {
        g->apply_ctas = ctas * sms;
        if ((rc = build_items(g, toff, cand_items[ii])) != FFT_OK) return false;
        if (tried == 0 || last < 20.0) {
            if ((rc = launch_JT(g, d, out_v, st)) != FFT_OK) return false;
            if ((rc = launch_J(g, m, out_m, st)) != FFT_OK) return false;
        }
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess && (rc = launch_JT(g, d, out_v, st)) != FFT_OK) return false;
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess && (rc = launch_J(g, m, out_m, st)) != FFT_OK) return false;
        if (e == cudaSuccess) e = cudaEventRecord(e2, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e2);
        float ms_jt = 0.0f, ms_j = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_jt, e0, e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_j, e1, e2);
        if (e != cudaSuccess) return false;
        ++tried;
        last = (double)ms_j + ms_jt;
        if (last < best) {
            best = last;
            best_j = ms_j;
            best_jt = ms_jt;
            best_items = cand_items[ii];
            best_ii = ii;
            best_ctas = ctas;
        }
        return true;
    };
    if (e == cudaSuccess) {
        int worse = 0;
        for (int ii = 0; ii < n_cand; ++ii) {
            if (!try_one(occ, ii)) break;
            worse = (last > 1.02 * best) ? worse + 1 : 0;
            if (worse == 2) break;
        }
        if (e == cudaSuccess && rc == FFT_OK && occ > 1) {
            const int centre = best_ii;
            for (int ii = std::max(0, centre - 1); ii <= std::min(n_cand - 1, centre + 1); ++ii)
                if (!try_one(occ - 1, ii)) break;
        }
    }
    if (e == cudaSuccess && rc == FFT_OK) {
        g->apply_ctas = best_ctas * sms;
        rc = build_items(g, toff, best_items);
    }
    if (e == cudaSuccess && rc == FFT_OK) e = cudaStreamSynchronize(st);
    cudaFree(m);
    cudaFree(d);
    cudaFree(out_v);
    cudaFree(out_m);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    if (rc != FFT_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fft_geom_autotune");
    if (info) {
        info->items_per_cta = best_items;
        info->ctas_per_sm = best_ctas;
        info->ms_J = best_j;
        info->ms_JT = best_jt;
        info->n_tried = tried;
    }
    return FFT_OK;
}
