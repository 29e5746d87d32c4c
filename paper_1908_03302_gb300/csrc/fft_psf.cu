// Hessian point-spread functions H_S e_k = J_S^T J_S e_k (Sec. II-D, Eq. resolution_2): the
// misfit Hessian applied to a unit perturbation at voxel k, restricted to a subset S of rows
// (a ring subset of the acquisition).
//
// FP32 CUDA-core path: column k of J_S is evaluated row by row (one thread per row of S),
// then J^T is applied to it. J^T skips rows whose weight is zero, so the cost of each PSF
// follows the rows whose support holds the spike.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
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
    D[p] = phi_lookup_global(vv, tab + (int64_t)b * n_tab, n_tab) * (is * ir) * r.b.w;
}

struct DParams {
    const RowRec* rec;
    const int32_t* row_band;
    const BandConst* bc;
    const float2* tab;
    int n_tab;
    const RowRec64* rec64;
    double ox, oy, oz, h;
    int nx, ny;
    const int64_t* spikes;    // spikes of this block
    int n_k;                  // spikes in the block
    const uint8_t* grp;       // group of each row (0xFF: in no subset)
    int64_t M;
    bool naive;
};

// Sparse rows of D for a block of spikes, one entry per spike k with J[p, spike_k] != 0 for the
// rows in some subset: k in bits 0-15 and the BF16 of C_p J[p, spike_k] in bits 16-31 (the
// tensor-core kernel's B operand; its A tile holds J / C_p). COUNT pass writes cnt[p], FILL
// pass writes at off[p].
template <bool FILL>
__global__ void dsparse_kernel(const DParams D, int32_t* __restrict__ cnt, const int64_t* __restrict__ off,
                               uint32_t* __restrict__ ent) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= D.M) return;
    if (D.grp[p] == 0xFF) {
        if (!FILL) cnt[p] = 0;
        return;
    }
    const RowRec r = D.rec[p];
    const int b = D.row_band[p];
    const BandConst c = D.bc[b];
    int n = 0;
    int64_t o = FILL ? off[p] : 0;
    for (int k = 0; k < D.n_k; ++k) {
        const int64_t v = D.spikes[k];
        const int ix = (int)(v % D.nx), iy = (int)((v / D.nx) % D.ny), iz = (int)(v / ((int64_t)D.nx * D.ny));
        const float jv = jentry_f32(r, c, D.tab + (int64_t)b * D.n_tab, D.n_tab, D.rec64, (int)p, D.ox, D.oy, D.oz,
                                    D.h, ix, iy, iz, D.naive);
        if (jv == 0.0f) continue;
        if (FILL)
            ent[o + n] = (uint32_t)k |
                         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(jv * r.b.w)) << 16);
        ++n;
    }
    if (!FILL) cnt[p] = n;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

// Host only: rows grouped by the set of subsets that hold them (see fft_gb300.h).
extern "C" fft_status fft_psf_row_groups(int64_t n_rows, const int32_t* subset_off, int32_t n_subsets,
                                         const int32_t* subset_rows, uint8_t* grp, uint32_t* gmask,
                                         int32_t* n_groups) {
    FFT_ARG(subset_off && grp && gmask && n_groups, "fft_psf_row_groups: null argument");
    FFT_ARG(n_rows >= 0 && n_subsets >= 1 && n_subsets <= 32, "fft_psf_row_groups: need n_rows >= 0 and 1 .. 32 subsets");
    FFT_ARG(subset_off[0] == 0, "fft_psf_row_groups: subset_off[0] must be 0");
    for (int s = 0; s < n_subsets; ++s)
        FFT_ARG(subset_off[s + 1] >= subset_off[s], "fft_psf_row_groups: subset offsets must be non-decreasing");
    FFT_ARG(subset_off[n_subsets] == 0 || subset_rows, "fft_psf_row_groups: null subset_rows");
    std::vector<uint32_t> member((size_t)n_rows, 0u);
    for (int s = 0; s < n_subsets; ++s)
        for (int32_t i = subset_off[s]; i < subset_off[s + 1]; ++i) {
            const int32_t p = subset_rows[i];
            FFT_ARG(p >= 0 && p < n_rows, "fft_psf_row_groups: subset row out of range");
            FFT_ARG(!((member[p] >> s) & 1u), "fft_psf_batch: a subset lists a row twice");
            member[p] |= 1u << s;
        }
    int32_t ng = 0;
    for (int64_t p = 0; p < n_rows; ++p) {
        grp[p] = 0xFF;
        if (!member[p]) continue;
        int32_t gi = 0;
        while (gi < ng && gmask[gi] != member[p]) ++gi;
        if (gi == ng) {
            if (ng == PSF_TC_MAX_GROUPS) {   // too many distinct sets for one launch
                *n_groups = -1;
                return FFT_OK;
            }
            gmask[ng++] = member[p];
        }
        grp[p] = (uint8_t)gi;
    }
    *n_groups = ng;
    return FFT_OK;
}

namespace {

// Tensor-core path for subsets whose rows fall into at most PSF_TC_MAX_GROUPS groups (rows with
// the same set of subsets holding them): D = J E for blocks of spikes, one launch per block.
// out_dev is the output of subsets [0, n_subsets) with n_spike spikes each.
fft_status psf_tc_groups(fft_geom g, const int64_t* spike_vox, int32_t n_spike, int32_t n_subsets,
                         const std::vector<uint8_t>& grp, const std::vector<uint32_t>& gmask, float* out_dev,
                         cudaStream_t st) {
    const int n_groups = (int)gmask.size();
    const int max_k = psf_tc_max_spikes(g, n_groups);
    if (max_k < 1) {
        set_error("fft_psf_batch: the tensor-core tiles do not fit in shared memory with these tables");
        return FFT_ERR_ARG;
    }
    const int k_blk = std::min<int>(max_k, n_spike);
    uint8_t* d_grp = nullptr;
    int32_t* d_cnt = nullptr;
    int64_t* d_off = nullptr;
    int64_t* d_spk = nullptr;
    uint32_t* d_ent = nullptr;
    fft_status rc = FFT_OK;
    cudaError_t e = cudaMalloc(&d_grp, g->M);
    if (e == cudaSuccess) e = cudaMalloc(&d_cnt, sizeof(int32_t) * g->M);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int64_t) * (g->M + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_spk, sizeof(int64_t) * n_spike);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_grp, grp.data(), g->M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_spk, spike_vox, sizeof(int64_t) * n_spike, cudaMemcpyHostToDevice, st);
    std::vector<int32_t> cnt(g->M);
    std::vector<int64_t> off(g->M + 1);
    for (int k0 = 0; k0 < n_spike && e == cudaSuccess && rc == FFT_OK; k0 += k_blk) {
        const int nk = std::min(k_blk, n_spike - k0);
        DParams D;
        D.rec = g->rec;
        D.row_band = g->row_band;
        D.bc = g->d_band;
        D.tab = g->tab;
        D.n_tab = g->n_tab;
        D.rec64 = g->rec64;
        D.ox = g->grid.origin[0];
        D.oy = g->grid.origin[1];
        D.oz = g->grid.origin[2];
        D.h = g->grid.h;
        D.nx = g->grid.nx;
        D.ny = g->grid.ny;
        D.spikes = d_spk + k0;
        D.n_k = nk;
        D.grp = d_grp;
        D.M = g->M;
        D.naive = (g->dt_mode == FFT_DT_NAIVE);
        const unsigned blocks = (unsigned)ceil_div(g->M, 128);
        dsparse_kernel<false><<<blocks, 128, 0, st>>>(D, d_cnt, nullptr, nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * g->M, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        off[0] = 0;
        for (int64_t p = 0; p < g->M; ++p) off[p + 1] = off[p] + cnt[p];
        const int64_t nnz = off[g->M];
        if (nnz > (int64_t)UINT32_MAX) {   // the kernel keeps 32-bit offsets into D
            rc = FFT_ERR_ARG;
            set_error("fft_psf_batch: more than 2^32 - 1 non-zeros in one block of D; use fewer spikes per call");
            break;
        }
        if (nnz == 0) continue;
        cudaFree(d_ent);
        d_ent = nullptr;
        e = cudaMalloc(&d_ent, sizeof(uint32_t) * nnz);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (g->M + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            dsparse_kernel<true><<<blocks, 128, 0, st>>>(D, nullptr, d_off, d_ent);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            rc = launch_psf_tc(g, d_off, d_ent, d_grp, n_groups, gmask.data(), n_subsets, n_spike, k0, nk, out_dev, st);
    }
    cudaFree(d_grp);
    cudaFree(d_cnt);
    cudaFree(d_off);
    cudaFree(d_spk);
    cudaFree(d_ent);
    if (rc != FFT_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fft_psf_batch (tensor cores)");
    return FFT_OK;
}

// Tensor-core path. Rows are grouped by the set of subsets that hold them (for nested subsets
// one group per subset); with more than PSF_TC_MAX_GROUPS distinct sets the subsets are taken
// one at a time.
fft_status psf_tc_path(fft_geom g, const int64_t* spike_vox, int32_t n_spike, const int32_t* subset_off,
                       int32_t n_subsets, const int32_t* subset_rows, float* out_dev, cudaStream_t st) {
    // rows listed twice are rejected here, before any device work
    std::vector<uint8_t> grp(g->M);
    std::vector<uint32_t> gmask(PSF_TC_MAX_GROUPS);
    int32_t n_groups = 0;
    fft_status rc = fft_psf_row_groups(g->M, subset_off, n_subsets, subset_rows, grp.data(), gmask.data(), &n_groups);
    if (rc != FFT_OK) return rc;
    const bool fits = n_groups >= 0;
    gmask.resize(fits ? n_groups : 0);
    g->psf_tc_mma_flops = 0.0;
    g->psf_tc_entries = 0.0;
    cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(float) * (size_t)n_subsets * n_spike * g->V, st);
    if (e != cudaSuccess) return cuda_fail(e, "fft_psf_batch (tensor cores)");
    if (fits && gmask.empty()) return FFT_OK;
    if (fits) return psf_tc_groups(g, spike_vox, n_spike, n_subsets, grp, gmask, out_dev, st);
    for (int s = 0; s < n_subsets; ++s) {
        std::fill(grp.begin(), grp.end(), (uint8_t)0xFF);
        for (int32_t i = subset_off[s]; i < subset_off[s + 1]; ++i) grp[subset_rows[i]] = 0;
        if (subset_off[s + 1] == subset_off[s]) continue;
        const std::vector<uint32_t> one(1, 1u);
        rc = psf_tc_groups(g, spike_vox, n_spike, 1, grp, one, out_dev + (int64_t)s * n_spike * g->V, st);
        if (rc != FFT_OK) return rc;
    }
    return FFT_OK;
}

// FP32 path with the four-column J^T: the columns of D = J_S E are taken in (spike, subset)
// order, so that a group of four mostly holds one spike's nested subsets and their rows are
// evaluated once for all of them; each group is one column evaluation per member and one
// four-column J^T into a staging block, copied to its outputs.
fft_status psf_fp32_batched(fft_geom g, const int64_t* spike_vox, int32_t n_spike, const int32_t* subset_off,
                            int32_t n_subsets, const int32_t* d_rows, float* out_dev, cudaStream_t st) {
    float* D4 = nullptr;
    float* Y4 = nullptr;
    cudaError_t e = cudaMalloc(&D4, sizeof(float) * 4 * g->M);
    if (e == cudaSuccess) e = cudaMalloc(&Y4, sizeof(float) * 4 * g->V);
    fft_status rc = FFT_OK;
    const int64_t n_cols = (int64_t)n_spike * n_subsets;
    const double3 o64 = make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]);
    for (int64_t c0 = 0; c0 < n_cols && e == cudaSuccess && rc == FFT_OK; c0 += 4) {
        const int nc = (int)std::min<int64_t>(4, n_cols - c0);
        e = cudaMemsetAsync(D4, 0, sizeof(float) * 4 * g->M, st);
        for (int j = 0; j < nc && e == cudaSuccess; ++j) {
            const int k = (int)((c0 + j) / n_subsets), s = (int)((c0 + j) % n_subsets);
            const int32_t a = subset_off[s], n = subset_off[s + 1] - a;
            if (n == 0) continue;
            if (g->dt_mode == FFT_DT_NAIVE)
                column_kernel<FFT_DT_NAIVE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                    g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                    spike_vox[k], g->rec64, o64, g->grid.h, D4 + (int64_t)j * g->M);
            else
                column_kernel<FFT_DT_STABLE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                    g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                    spike_vox[k], g->rec64, o64, g->grid.h, D4 + (int64_t)j * g->M);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        if ((rc = launch_JT_batch(g, D4, 4, Y4, st)) != FFT_OK) break;
        for (int j = 0; j < nc && e == cudaSuccess; ++j) {
            const int k = (int)((c0 + j) / n_subsets), s = (int)((c0 + j) % n_subsets);
            e = cudaMemcpyAsync(out_dev + ((int64_t)s * n_spike + k) * g->V, Y4 + (int64_t)j * g->V,
                                sizeof(float) * g->V, cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(D4);
    cudaFree(Y4);
    if (rc != FFT_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "fft_psf_batch (four-column FP32)");
    if (e2 != cudaSuccess) return cuda_fail(e2, "fft_psf_batch (four-column FP32) sync");
    return FFT_OK;
}

}  // namespace

extern "C" fft_status fft_psf_batch(fft_geom g, const int64_t* spike_vox, int32_t n_spike,
                                    const int32_t* subset_off, int32_t n_subsets, const int32_t* subset_rows,
                                    int32_t mode, float* out_dev, void* stream) {
    FFT_API_RANGE("fft_psf_batch");
    FFT_ARG(g && spike_vox && subset_off && out_dev, "fft_psf_batch: null argument");
    FFT_ARG(n_spike >= 1 && n_subsets >= 1, "fft_psf_batch: need at least one spike and one subset");
    FFT_ARG(mode >= 0 && mode <= 2,
            "fft_psf_batch: mode must be 0 (FP32), 1 (BF16 tensor cores) or 2 (FP32, four columns per J^T)");
    FFT_ARG(mode == 0 || n_subsets <= 32, "fft_psf_batch: the tensor-core path takes at most 32 subsets");
    FFT_ARG(g->phi_kind == PHI_TABLE, "fft_psf_batch: needs a geometry built from sampled tables (not sine series)");
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
    if (mode == 1) {   // (rows listed twice in a subset are rejected there, before any device work)
        rc = psf_tc_path(g, spike_vox, n_spike, subset_off, n_subsets, subset_rows, out_dev, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (rc != FFT_OK) return rc;
        if (e2 != cudaSuccess) return cuda_fail(e2, "fft_psf_batch sync");
        return FFT_OK;
    }
    int32_t* d_rows = nullptr;
    FFT_CUDA(cudaMalloc(&d_rows, sizeof(int32_t) * (n_idx > 0 ? n_idx : 1)));
    cudaError_t e = cudaSuccess;
    if (n_idx > 0) e = cudaMemcpyAsync(d_rows, subset_rows, sizeof(int32_t) * n_idx, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && mode == 2) {
        rc = psf_fp32_batched(g, spike_vox, n_spike, subset_off, n_subsets, d_rows, out_dev, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFree(d_rows);
        if (rc != FFT_OK) return rc;
        if (e2 != cudaSuccess) return cuda_fail(e2, "fft_psf_batch sync");
        return FFT_OK;
    }
    float* D = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&D, sizeof(float) * g->M);
    if (e != cudaSuccess) {
        cudaFree(d_rows);
        return cuda_fail(e, "fft_psf_batch cudaMalloc");
    }
    for (int s = 0; s < n_subsets && e == cudaSuccess && rc == FFT_OK; ++s) {
        const int32_t a = subset_off[s], n = subset_off[s + 1] - a;
        for (int k = 0; k < n_spike && e == cudaSuccess && rc == FFT_OK; ++k) {
            e = cudaMemsetAsync(D, 0, sizeof(float) * g->M, st);
            if (e != cudaSuccess) break;
            if (n > 0) {
                const double3 o64 = make_double3(g->grid.origin[0], g->grid.origin[1], g->grid.origin[2]);
                if (g->dt_mode == FFT_DT_NAIVE)
                    column_kernel<FFT_DT_NAIVE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                        g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                        spike_vox[k], g->rec64, o64, g->grid.h, D);
                else
                    column_kernel<FFT_DT_STABLE><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
                        g->rec, g->row_band, g->d_band, g->tab, g->n_tab, d_rows + a, n, g->grid.nx, g->grid.ny,
                        spike_vox[k], g->rec64, o64, g->grid.h, D);
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
