// Internal definitions shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fft_gb300.h"

namespace fftgb {

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string& msg);
fft_status cuda_fail(cudaError_t e, const char* what);

#define FFT_CUDA(call)                                         \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::fftgb::cuda_fail(_e, #call); \
    } while (0)

#define FFT_ARG(cond, msg)                  \
    do {                                    \
        if (!(cond)) {                      \
            ::fftgb::set_error(msg);        \
            return FFT_ERR_ARG;             \
        }                                   \
    } while (0)

// ------------------------------------------------------------------ tracing
// An NVTX range named after the C-ABI call around its body, so that profiler timelines and
// `ncu --nvtx --nvtx-include "<name>/"` can pick out the kernels of one call. Without a
// profiler attached the push and pop cost a function call each.
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};
#define FFT_API_RANGE(name) ::fftgb::ApiRange fft_api_range_(name)

// ------------------------------------------------------------------ tiling constants
// A tile is 16 x 16 x 8 voxels handled by one CTA of 8 warps. Warp w owns the 8 x 8 x 4
// region at (8 (w & 1), 8 ((w >> 1) & 1), 4 (w >> 2)), split into two 8 x 4 x 4 sub-bricks
// stacked in y. Lane l owns the 4 consecutive x voxels at
// (4 (l & 1), (l >> 1) & 3, l >> 3) of a sub-brick.
constexpr int TILE_X = 16, TILE_Y = 16, TILE_Z = 8;
constexpr int TILE_VOX = TILE_X * TILE_Y * TILE_Z;
constexpr int APPLY_WARPS = 8;
constexpr int APPLY_THREADS = APPLY_WARPS * 32;
constexpr int NX_LANE = 4;             // voxels per lane per sub-brick (along x)
constexpr int SUBS_PER_WARP = 2;
constexpr int MAX_BANDS = 8;
constexpr int DEFAULT_ITEMS_PER_CTA = 8;   // work items per persistent CTA before tuning
constexpr float CULL_MARGIN = 2e-3f;   // in units of the band's maximum detour

// Per-row record, lengths in units of the row's band maximum detour U_b = c0 * dt_max_b.
struct RowRec {
    float4 a;   // (o_x, o_y, o_z, hl): pair midpoint, half pair length
    float4 b;   // (e_x, e_y, e_z, C): unit axis, C = -L h^3 / (2 pi c0^3 U_b^2) (SI seconds per m/s per
                // unit Phi / (R_xs R_xr) in band units)
};

// Per-row FP64 record used by the FP64 detour mode (SI metres).
struct RowRec64 {
    double xs[3];
    double xr[3];
};

struct BandConst {
    float h;          // voxel spacing in band units
    float org[3];     // grid origin in band units
    double U;         // band unit length in metres (c0 * dt_max)
    int32_t sharp;    // Phi just below the cut-off is not negligible: decide the cut in FP64
    int32_t pad;
};

// Half-width (in units of the band's maximum detour) of the band around the cut-off inside
// which a sharp band re-decides "dt < dt_max" in FP64. The FP32 detour near the cut-off is
// good to ~5e-7 (FP64-derived entry bases, approximate rsqrt / rcp), so 2e-6 keeps a 4x margin.
constexpr float CUT_BAND = 2e-6f;

// Representation of Phi inside the kernels.
enum { PHI_TABLE = 0,   // sampled table, linear interpolation (fft_table_build)
       PHI_TRIG = 1 };  // sine series, Clenshaw recurrence (fft_trig_build)
constexpr int TRIG_MAX_TERMS = 256;

// Work item: rows [e0, e1) of tile `tile`'s entry list; J^T writes to slot `slot` of the
// partial buffer when the tile has several items, else (slot < 0) straight to g.
struct Item {
    int32_t tile;
    int32_t slot;
    int64_t e0, e1;
};

}  // namespace fftgb

// ------------------------------------------------------------------ handles
struct fft_table_s {
    int dev;
    int32_t n;                 // samples (table) or terms (series)
    double dt_max;
    double* d_phi;             // table: device FP64 samples [n]; series: nullptr
    int32_t kind = 0;          // fftgb::PHI_TABLE or fftgb::PHI_TRIG
    double dw = 0.0;           // series: node spacing (rad/s)
    std::vector<double> coef;  // series: a_1 .. a_n (host, FP64)
};

struct fft_geom_s {
    int dev;
    int64_t M;
    int64_t V;
    int32_t n_tx;
    fft_grid grid;
    double c0;
    int32_t n_bands;
    int32_t n_tab;
    int32_t dt_mode;
    int32_t phi_kind = 0;                // fftgb::PHI_TABLE or fftgb::PHI_TRIG (all bands alike)
    int32_t trig_nq = 0;                 // series: coefficient groups of 4 per band (padded)
    int32_t trig_terms = 0;              // series: the largest term count over the bands
    double psf_tc_mma_flops = 0.0;       // MMA flops of the last tensor-core fft_psf_batch call
    double psf_tc_entries = 0.0;         // J entries it generated
    bool guard;                          // a (virtual) voxel centre coincides with a transducer
    bool sharp = false;                  // some band's Phi does not vanish at its cut-off
    fftgb::BandConst band[fftgb::MAX_BANDS];
    double dt_max[fftgb::MAX_BANDS];
    // device arrays
    fftgb::BandConst* d_band = nullptr;  // [n_bands]
    fftgb::RowRec* rec = nullptr;        // [M]
    fftgb::RowRec64* rec64 = nullptr;    // [M] (FP64 mode only)
    int32_t* row_band = nullptr;         // [M]
    float2* tab = nullptr;               // [n_bands * n_tab] (Phi_k, Phi_{k+1} - Phi_k)
    int32_t tiles[3];
    int64_t n_tiles = 0;
    int64_t E = 0;                       // entries
    int64_t* tile_off = nullptr;         // [n_tiles + 1]
    int32_t* tile_rows = nullptr;        // [E]
    float4* ebase = nullptr;             // [E] (p + hl, p - hl, c1, c2) of the tile origin in the row's pair frame
    float* ebase3 = nullptr;             // [E] c3 of the tile origin
    int64_t* row_off = nullptr;          // [M + 1]
    int64_t* row_ent = nullptr;          // [E] tile-major entry ids of each row, ascending
    fftgb::Item* items = nullptr;        // [n_items]
    int32_t n_items = 0;
    int32_t n_slots = 0;
    int32_t* tile_slot0 = nullptr;       // [n_tiles] first slot of a multi-item tile, -1 single, -2 none
    int32_t* tile_nslot = nullptr;       // [n_tiles]
    float* jpart = nullptr;              // [E * 4]
    float* gpart = nullptr;              // [n_slots * TILE_VOX]
    int32_t* counter = nullptr;          // [4] work counters
    int64_t support = 0;
    int64_t evaluated = 0;
    double frob2 = -1.0;
    int64_t scratch_bytes = 0;
    int apply_ctas = 0;                  // persistent grid of the apply kernels (8-warp CTAs)
    int sharp_warps = 8;                 // warps per CTA of the sharp-band single-column kernels
    int sharp_ctas = 0;                  // their persistent grid
    int plain_warps = 8;                 // warps per CTA of the plain stable-detour table kernels
    int plain_ctas = 0;                  // their persistent grid when plain_warps > 8
    // Sharp geometries split each tile's entries: rows of bands whose Phi vanishes at the cut
    // first, then rows of sharp bands; items never mix the two, the plain items come first.
    std::vector<int64_t> tile_nplain;    // host: plain entries of each tile (empty: no split)
    int32_t n_items_plain = 0;           // items [0, n_items_plain) hold plain rows only
    int items_per_cta = 0;               // work-item granularity (autotuned or the default)
    // CG workspace (allocated on first use)
    float* cg_r = nullptr;               // [M] residual d - J m
    float* cg_q = nullptr;               // [M] J p
    float* cg_s = nullptr;               // [V] J^T r - lambda m
    float* cg_p = nullptr;               // [V] search direction
    float* cg_d = nullptr;               // [M] copy of the data
    float* cg_m = nullptr;               // [V] iterate
    double* cg_scal = nullptr;           // [8] device scalars
    double* cg_dots = nullptr;           // [2 * DOT_BLOCKS] partial inner products
    int32_t* cg_status = nullptr;        // [1]
    float* vol = nullptr;                // [V] volume scratch of the 2-D apply (allocated on first use)
    float4* psf_crec = nullptr;          // candidate records of the tensor-core PSF path (grow-only)
    int64_t psf_crec_cap = 0;            // its capacity in candidates (3 float4 each)
    float* jpart4 = nullptr;             // [E * 8 * 4] J partials of the four-column apply (first use)
    float* gpart4 = nullptr;             // [n_slots * 4 * TILE_VOX] J^T partials of the four-column apply
    double* cg_hist = nullptr;           // [cg_hist_cap]
    int32_t cg_hist_cap = 0;
    void* cg_graph = nullptr;            // cudaGraphExec_t of the iteration loop
    int32_t cg_graph_iters = -1;
    void* cg_graph_cont = nullptr;       // cudaGraphExec_t of a continued loop (fft_cg_continue)
    int32_t cg_graph_cont_iters = -1;
    int64_t cg_done = -1;                // iterations behind the handle's CG state (-1: no state)
    void* cg_stream = nullptr;           // private capture stream
};

namespace fftgb {
// Launch helpers implemented in fft_apply.cu (used by CG and PSF).
fft_status launch_J(fft_geom g, const float* m, float* d, cudaStream_t st);
fft_status launch_JT(fft_geom g, const float* din, float* gout, cudaStream_t st);
fft_status launch_J_batch(fft_geom g, const float* m, int n, float* d, cudaStream_t st);
fft_status build_items(fft_geom g, const std::vector<int64_t>& toff, int items_per_cta);
fft_status launch_JT_batch(fft_geom g, const float* din, int n, float* gout, cudaStream_t st);
fft_status launch_JT_rows(fft_geom g, const float* din, float* gout, cudaStream_t st);
fft_status check_device(int dev);
fft_status count_support(fft_geom g, int64_t* support, int64_t* evaluated);
fft_status compute_frob2(fft_geom g, double* out);
fft_status set_apply_attributes(fft_geom g);
int apply_occupancy(fft_geom g);
size_t apply_smem(fft_geom g);
void sharp_launch_shape(fft_geom g);
void plain_launch_shape(fft_geom g);
// Tensor-core PSFs: rows are grouped by the set of subsets that hold them (at most
// PSF_TC_MAX_GROUPS distinct sets per launch).
constexpr int PSF_TC_MAX_GROUPS = 32;
int psf_tc_max_spikes(fft_geom g, int n_groups);
fft_status launch_psf_tc(fft_geom g, const int64_t* d_off, const uint32_t* d_ent, const uint8_t* grp, int n_groups,
                         const uint32_t* gmask, int n_sub, int n_spike, int k0, int nk, float* out, cudaStream_t st);
int64_t ceil_div(int64_t a, int64_t b);
// Resolve (and so load) the no-allocation PSF's static scratch on device `dev` (current).
fft_status noalloc_prepare(int dev);
}  // namespace fftgb
