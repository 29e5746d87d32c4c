// Geometry set-up: per-row records, band tables in the device layout, and the culled
// (tile, row) lists that make the truncated operator sparse (Sec. II-C: truncating the
// maximum detour controls the sparsity of F).
//
// A (tile, row) entry is kept unless a lower bound of the detour over the tile's voxel
// centres is >= the band's cut-off: R is convex, so its tangent plane at the tile centre
// bounds it from below over the tile. The tile-major lists are built by one CTA per tile
// scanning all rows (rows ascending, so the order is deterministic); the row-major view
// used by the J reduction is the same set, grouped by row with entries in ascending order.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft_common.cuh"
#include "fft_device.cuh"

namespace fftgb {

namespace {

constexpr int CULL_THREADS = 256;

struct CullParams {
    const RowRec* rec;
    const int32_t* row_band;
    const BandConst* bc;
    int64_t M;
    int tiles_x, tiles_y;
    int nx, ny, nz;
};

__device__ __forceinline__ bool tile_keeps_row(const CullParams& C, int T, int64_t p) {
    const int tx = T % C.tiles_x, ty = (T / C.tiles_x) % C.tiles_y, tz = T / (C.tiles_x * C.tiles_y);
    const RowRec r = C.rec[p];
    const BandConst bc = C.bc[C.row_band[p]];
    const float hb = bc.h;
    const float cx = fmaf((float)(TILE_X * tx) + 0.5f * (TILE_X - 1), hb, bc.org[0]) - r.a.x;
    const float cy = fmaf((float)(TILE_Y * ty) + 0.5f * (TILE_Y - 1), hb, bc.org[1]) - r.a.y;
    const float cz = fmaf((float)(TILE_Z * tz) + 0.5f * (TILE_Z - 1), hb, bc.org[2]) - r.a.z;
    if (!box_may_touch(cx, cy, cz, r.b.x, r.b.y, r.b.z, r.a.w, 0.5f * (TILE_X - 1) * hb,
                       0.5f * (TILE_Y - 1) * hb, 0.5f * (TILE_Z - 1) * hb))
        return false;
    // keep the row only if one of the tile's 16 sub-bricks (8 x 4 x 4, the apply kernels'
    // culling unit) inside the grid may reach the support: rows that reach none of them
    // would be staged by every region for nothing
    const float x0 = cx - 0.5f * (TILE_X - 1) * hb, y0 = cy - 0.5f * (TILE_Y - 1) * hb,
                z0 = cz - 0.5f * (TILE_Z - 1) * hb;
    for (int sb = 0; sb < 16; ++sb) {
        const int sx = 8 * (sb & 1), sy = 4 * ((sb >> 1) & 3), sz = 4 * (sb >> 3);
        if (TILE_X * tx + sx >= C.nx || TILE_Y * ty + sy >= C.ny || TILE_Z * tz + sz >= C.nz) continue;
        if (box_may_touch(fmaf((float)sx + 3.5f, hb, x0), fmaf((float)sy + 1.5f, hb, y0),
                          fmaf((float)sz + 1.5f, hb, z0), r.b.x, r.b.y, r.b.z, r.a.w, 3.5f * hb, 1.5f * hb,
                          1.5f * hb))
            return true;
    }
    return false;
}

// Kept rows of tile T (cnt), and of those the rows of bands that are not sharp (cnt_plain,
// nullable; counted only when `split`).
__global__ void tile_count_kernel(const CullParams C, int split, int64_t* __restrict__ cnt,
                                  int64_t* __restrict__ cnt_plain) {
    __shared__ int64_t sh[2][CULL_THREADS / 32];
    const int T = blockIdx.x;
    int64_t c = 0, cp = 0;
    for (int64_t p = threadIdx.x; p < C.M; p += CULL_THREADS) {
        if (tile_keeps_row(C, T, p)) {
            ++c;
            if (split && !C.bc[C.row_band[p]].sharp) ++cp;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        cp += __shfl_xor_sync(0xffffffffu, cp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = c;
        sh[1][threadIdx.x >> 5] = cp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0, sp = 0;
        for (int w = 0; w < CULL_THREADS / 32; ++w) {
            s += sh[0][w];
            sp += sh[1][w];
        }
        cnt[T] = s;
        if (cnt_plain) cnt_plain[T] = sp;
    }
}

// Writes the kept rows of tile T in ascending row order; with `split` (nplain given) the rows of
// bands that are not sharp first (from off[T]) and the rows of sharp bands after them (from
// off[T] + nplain[T]), each part in ascending row order.
__global__ void tile_fill_kernel(const CullParams C, const int64_t* __restrict__ off,
                                 const int64_t* __restrict__ nplain, int32_t* __restrict__ rows) {
    __shared__ int wsum[2][CULL_THREADS / 32];
    const int T = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t base0 = off[T], base1 = nplain ? off[T] + nplain[T] : off[T + 1];
    for (int64_t p0 = 0; p0 < C.M; p0 += CULL_THREADS) {
        const int64_t p = p0 + threadIdx.x;
        const bool keep = p < C.M && tile_keeps_row(C, T, p);
        const bool sharp = keep && nplain && C.bc[C.row_band[p]].sharp;
        const uint32_t bal0 = __ballot_sync(0xffffffffu, keep && !sharp);
        const uint32_t bal1 = __ballot_sync(0xffffffffu, sharp);
        if (lane == 0) {
            wsum[0][warp] = __popc(bal0);
            wsum[1][warp] = __popc(bal1);
        }
        __syncthreads();
        int before0 = 0, total0 = 0, before1 = 0, total1 = 0;
        for (int w = 0; w < CULL_THREADS / 32; ++w) {
            if (w < warp) {
                before0 += wsum[0][w];
                before1 += wsum[1][w];
            }
            total0 += wsum[0][w];
            total1 += wsum[1][w];
        }
        const uint32_t below = (1u << lane) - 1u;
        if (keep) {
            const int64_t pos = sharp ? base1 + before1 + __popc(bal1 & below) : base0 + before0 + __popc(bal0 & below);
            if (pos < off[T + 1]) rows[pos] = (int32_t)p;
        }
        base0 += total0;
        base1 += total1;
        __syncthreads();
    }
}

// FP64 pair-frame coordinates of each entry's tile origin (voxel (TX, TY, TZ) centre) in band
// units: p = (x_T - o).e and c = (x_T - o) x e. Computing them here in double precision keeps
// the large (~L/2) coordinates out of FP32 arithmetic; the kernels add only small offsets.
__global__ void entry_base_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ rows_of_entry,
                                  const double* __restrict__ tx, const int32_t* __restrict__ pairs,
                                  const int32_t* __restrict__ row_band, const BandConst* __restrict__ bc,
                                  double ox, double oy, double oz, double h, int tiles_x, int tiles_y,
                                  float4* __restrict__ ebase, float* __restrict__ ebase3) {
    const int T = blockIdx.x;
    const int tx_ = T % tiles_x, ty_ = (T / tiles_x) % tiles_y, tz_ = T / (tiles_x * tiles_y);
    const double xT = ox + (double)(TILE_X * tx_) * h;
    const double yT = oy + (double)(TILE_Y * ty_) * h;
    const double zT = oz + (double)(TILE_Z * tz_) * h;
    for (int64_t e = off[T] + threadIdx.x; e < off[T + 1]; e += blockDim.x) {
        const int p = rows_of_entry[e];
        const double* xs = tx + 3 * (int64_t)pairs[2 * p];
        const double* xr = tx + 3 * (int64_t)pairs[2 * p + 1];
        const double U = bc[row_band[p]].U;
        double ax = xr[0] - xs[0], ay = xr[1] - xs[1], az = xr[2] - xs[2];
        const double L = sqrt(ax * ax + ay * ay + az * az);
        ax /= L;
        ay /= L;
        az /= L;
        const double dx = (xT - 0.5 * (xs[0] + xr[0])) / U;
        const double dy = (yT - 0.5 * (xs[1] + xr[1])) / U;
        const double dz = (zT - 0.5 * (xs[2] + xr[2])) / U;
        const double pp = dx * ax + dy * ay + dz * az, hl = 0.5 * L / U;
        // p + hl and p - hl are the axial offsets from the emitter and the receiver; forming
        // them here keeps them exact when small (voxels near a transducer)
        ebase[e] = make_float4((float)(pp + hl), (float)(pp - hl), (float)(dy * az - dz * ay),
                               (float)(dz * ax - dx * az));
        ebase3[e] = (float)(dx * ay - dy * ax);
    }
}

__global__ void row_count_kernel(const int32_t* __restrict__ tile_rows, int64_t E, int32_t* __restrict__ cnt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < E) atomicAdd(&cnt[tile_rows[e]], 1);
}

__global__ void row_fill_kernel(const int32_t* __restrict__ tile_rows, int64_t E, const int64_t* __restrict__ row_off,
                                int32_t* __restrict__ cursor, int64_t* __restrict__ row_ent) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int p = tile_rows[e];
    int k = atomicAdd(&cursor[p], 1);
    row_ent[row_off[p] + k] = e;
}

// Insertion sort of each row's (short) entry list, so that its order does not depend on
// the order in which the fill kernel's atomics were served.
__global__ void row_sort_kernel(const int64_t* __restrict__ row_off, int64_t M, int64_t* __restrict__ row_ent) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    int64_t a = row_off[p], b = row_off[p + 1];
    for (int64_t i = a + 1; i < b; ++i) {
        int64_t x = row_ent[i], j = i - 1;
        while (j >= a && row_ent[j] > x) {
            row_ent[j + 1] = row_ent[j];
            --j;
        }
        row_ent[j + 1] = x;
    }
}

__global__ void pack_table_kernel(const double* __restrict__ phi, int n, float2* __restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    // Entry k holds (Phi_k - k dPhi_k, (n - 1) dPhi_k), dPhi_k = Phi_{k+1} - Phi_k, formed in FP64:
    // the interpolant on [k, k + 1) is then one FFMA in the normalised detour. The last entry
    // is the cut-off: Phi = 0 at and beyond dt_max (hard truncation), so it holds (0, 0).
    if (k == n - 1) {
        out[k] = make_float2(0.0f, 0.0f);
    } else {
        const double d = phi[k + 1] - phi[k];
        out[k] = make_float2((float)(phi[k] - (double)k * d), (float)(d * (double)(n - 1)));
    }
}

template <typename T>
fft_status dmalloc(fft_geom g, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("fft_geom_create: cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
        return FFT_ERR_OOM;
    }
    g->scratch_bytes += (int64_t)(count * sizeof(T));
    return FFT_OK;
}

void free_geom(fft_geom g) {
    if (!g) return;
    void* ptrs[] = {g->d_band, g->rec, g->rec64, g->row_band, g->tab, g->tile_off, g->tile_rows, g->ebase, g->ebase3,
                    g->row_off, g->row_ent, g->items, g->tile_slot0, g->tile_nslot, g->jpart,
                    g->gpart, g->counter, g->cg_r, g->cg_q, g->cg_s, g->cg_p, g->cg_d, g->cg_m,
                    g->cg_scal, g->cg_dots, g->cg_status, g->cg_hist, g->vol, g->jpart4, g->gpart4,
                    g->psf_crec};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->cg_graph) cudaGraphExecDestroy((cudaGraphExec_t)g->cg_graph);
    if (g->cg_graph_cont) cudaGraphExecDestroy((cudaGraphExec_t)g->cg_graph_cont);
    if (g->cg_stream) cudaStreamDestroy((cudaStream_t)g->cg_stream);
    delete g;
}

}  // namespace

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Work items: a tile's candidate rows in ranges of at most ch rows, ch chosen so that each
// persistent CTA sees about items_per_cta items (at least 64 rows, a multiple of 32); tiles
// split over several items write J^T partial slots. Heaviest items first. Replaces the
// geometry's previous items, slots and partial buffers (the J partials do not depend on them).
fft_status build_items(fft_geom g, const std::vector<int64_t>& toff, int items_per_cta) {
    const int64_t target = (int64_t)items_per_cta * g->apply_ctas;
    int64_t ch = std::max<int64_t>(64, ceil_div(std::max<int64_t>(g->E, 1), std::max<int64_t>(target, 1)));
    ch = ceil_div(ch, 32) * 32;
    // plain rows [toff, toff + nplain) and sharp-band rows [toff + nplain, toff1) of a split
    // geometry go to different items; the tile's slots number its plain items first
    const bool split = !g->tile_nplain.empty();
    std::vector<Item> items, items_sharp;
    std::vector<int32_t> slot0(g->n_tiles, -2), nslot(g->n_tiles, 0);
    int32_t slots = 0;
    for (int64_t T = 0; T < g->n_tiles; ++T) {
        const int64_t n = toff[T + 1] - toff[T];
        if (n == 0) continue;
        const int64_t np = split ? g->tile_nplain[T] : n;
        const int64_t kp = ceil_div(np, ch), ks = ceil_div(n - np, ch), k = kp + ks;
        if (k == 1) {
            (kp == 1 ? items : items_sharp).push_back(Item{(int32_t)T, -1, toff[T], toff[T + 1]});
            slot0[T] = -1;
        } else {
            slot0[T] = slots;
            nslot[T] = (int32_t)k;
            for (int64_t q = 0; q < k; ++q) {
                const int64_t lo = q < kp ? toff[T] : toff[T] + np, hi = q < kp ? toff[T] + np : toff[T + 1];
                const int64_t a = lo + (q < kp ? q : q - kp) * ch, b = std::min(hi, a + ch);
                (q < kp ? items : items_sharp).push_back(Item{(int32_t)T, slots + (int32_t)q, a, b});
            }
            slots += (int32_t)k;
        }
    }
    auto heavier = [](const Item& x, const Item& y) { return (x.e1 - x.e0) > (y.e1 - y.e0); };
    std::stable_sort(items.begin(), items.end(), heavier);
    std::stable_sort(items_sharp.begin(), items_sharp.end(), heavier);
    g->n_items_plain = (int32_t)items.size();
    items.insert(items.end(), items_sharp.begin(), items_sharp.end());
    if (g->items) {   // the buffers below are replaced: take them out of the scratch count
        g->scratch_bytes -= (int64_t)(sizeof(Item) * g->n_items + 2 * sizeof(int32_t) * g->n_tiles +
                                      sizeof(float) * (size_t)g->n_slots * TILE_VOX);
        if (g->jpart4)
            g->scratch_bytes -= (int64_t)(sizeof(float) * ((size_t)g->E * 32 + (size_t)g->n_slots * 4 * TILE_VOX));
    }
    void* old[] = {g->items, g->tile_slot0, g->tile_nslot, g->gpart, g->gpart4};
    for (void* q : old)
        if (q) cudaFree(q);
    g->items = nullptr;
    g->tile_slot0 = g->tile_nslot = nullptr;
    g->gpart = g->gpart4 = nullptr;
    if (g->jpart4) {   // the four-column scratch is rebuilt with the new slot count on first use
        cudaFree(g->jpart4);
        g->jpart4 = nullptr;
    }
    g->n_items = (int32_t)items.size();
    g->n_slots = slots;
    g->items_per_cta = items_per_cta;
    fft_status rc;
    if ((rc = dmalloc(g, &g->items, items.size())) != FFT_OK) return rc;
    if ((rc = dmalloc(g, &g->tile_slot0, g->n_tiles)) != FFT_OK) return rc;
    if ((rc = dmalloc(g, &g->tile_nslot, g->n_tiles)) != FFT_OK) return rc;
    if ((rc = dmalloc(g, &g->gpart, (size_t)slots * TILE_VOX)) != FFT_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (!items.empty()) e = cudaMemcpy(g->items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->tile_slot0, slot0.data(), sizeof(int32_t) * g->n_tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->tile_nslot, nslot.data(), sizeof(int32_t) * g->n_tiles, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "work items");
    // a captured CG loop holds the old item list: capture again on the next solve
    if (g->cg_graph) {
        cudaGraphExecDestroy((cudaGraphExec_t)g->cg_graph);
        g->cg_graph = nullptr;
        g->cg_graph_iters = -1;
    }
    if (g->cg_graph_cont) {
        cudaGraphExecDestroy((cudaGraphExec_t)g->cg_graph_cont);
        g->cg_graph_cont = nullptr;
        g->cg_graph_cont_iters = -1;
    }
    return FFT_OK;
}

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_geom_create(const double* tx_xyz, int32_t n_tx, const int32_t* rows,
                                      int64_t n_rows, const int32_t* band_of_row, const fft_grid* grid,
                                      double c0, const fft_table* tables, int32_t n_tables,
                                      int32_t dt_mode, fft_geom* out) {
    FFT_API_RANGE("fft_geom_create");
    FFT_ARG(out, "fft_geom_create: null out");
    *out = nullptr;
    FFT_ARG(tx_xyz && n_tx >= 2, "fft_geom_create: need at least two transducers");
    FFT_ARG(rows && n_rows >= 1 && n_rows < (int64_t)INT32_MAX, "fft_geom_create: need 1 .. 2^31-2 rows");
    FFT_ARG(grid && grid->nx >= 1 && grid->ny >= 1 && grid->nz >= 1 && grid->h > 0,
            "fft_geom_create: invalid grid");
    FFT_ARG(c0 > 0 && isfinite(c0), "fft_geom_create: c0 must be > 0");
    FFT_ARG(tables && n_tables >= 1 && n_tables <= MAX_BANDS, "fft_geom_create: need 1 .. 8 tables");
    FFT_ARG(dt_mode == FFT_DT_STABLE || dt_mode == FFT_DT_NAIVE || dt_mode == FFT_DT_FP64,
            "fft_geom_create: unknown dt_mode");
    int dev = 0;
    FFT_CUDA(cudaGetDevice(&dev));
    for (int b = 0; b < n_tables; ++b) {
        FFT_ARG(tables[b], "fft_geom_create: null table");
        FFT_ARG(tables[b]->kind == tables[0]->kind,
                "fft_geom_create: tables must be all sampled tables or all sine series");
        if (tables[0]->kind == PHI_TABLE)
            FFT_ARG(tables[b]->n == tables[0]->n, "fft_geom_create: all tables must have the same sample count");
        if (tables[b]->dev != dev) {
            set_error("fft_geom_create: table was built on another device");
            return FFT_ERR_STATE;
        }
    }
    const int32_t phi_kind = tables[0]->kind;
    FFT_ARG(phi_kind == PHI_TABLE || dt_mode == FFT_DT_STABLE,
            "fft_geom_create: sine-series tables need dt_mode FFT_DT_STABLE");
    // device layout of one band's Phi: n_tab float2 entries. Series: a 16-byte header (theta =
    // dw dt_max, the series argument at the cut-off) and the coefficients in groups of 4.
    int32_t trig_terms = 0;
    for (int b = 0; b < n_tables; ++b) trig_terms = std::max(trig_terms, tables[b]->n);
    const int32_t trig_nq = (trig_terms + 3) / 4;
    const int32_t n_tab = phi_kind == PHI_TABLE ? tables[0]->n : 2 + 2 * trig_nq;
    const int64_t V = (int64_t)grid->nx * grid->ny * grid->nz;
    FFT_ARG(V < ((int64_t)1 << 40), "fft_geom_create: grid too large");
    for (int64_t p = 0; p < n_rows; ++p) {
        int32_t s = rows[2 * p], r = rows[2 * p + 1];
        FFT_ARG(s >= 0 && s < n_tx && r >= 0 && r < n_tx, "fft_geom_create: row transducer index out of range");
        FFT_ARG(s != r, "fft_geom_create: a row has the same emitter and receiver");
        if (band_of_row)
            FFT_ARG(band_of_row[p] >= 0 && band_of_row[p] < n_tables, "fft_geom_create: band index out of range");
    }
    {
        int optin = 0;
        FFT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        size_t need = (((size_t)n_tables * n_tab * sizeof(float2) + 15) & ~(size_t)15) +
                      (size_t)APPLY_WARPS * 128 * sizeof(float4);
        if (need > (size_t)optin) {
            set_error("fft_geom_create: the tables (n_tables x n_samples x 8 bytes) do not fit in shared memory");
            return FFT_ERR_ARG;
        }
    }
    fft_geom g = new fft_geom_s();
    g->dev = dev;
    g->M = n_rows;
    g->V = V;
    g->n_tx = n_tx;
    g->grid = *grid;
    g->c0 = c0;
    g->n_bands = n_tables;
    g->n_tab = n_tab;
    g->dt_mode = dt_mode;
    g->phi_kind = phi_kind;
    g->trig_nq = phi_kind == PHI_TRIG ? trig_nq : 0;
    g->trig_terms = phi_kind == PHI_TRIG ? trig_terms : 0;
    g->guard = false;
    fft_status rc = FFT_OK;
#define GEOM_TRY(x)              \
    do {                         \
        rc = (x);                \
        if (rc != FFT_OK) {      \
            free_geom(g);        \
            return rc;           \
        }                        \
    } while (0)
#define GEOM_CUDA(x)                                 \
    do {                                             \
        cudaError_t _e = (x);                        \
        if (_e != cudaSuccess) {                     \
            rc = cuda_fail(_e, #x);                  \
            free_geom(g);                            \
            return rc;                               \
        }                                            \
    } while (0)

    // ---- bands
    std::vector<BandConst> hb(n_tables);
    for (int b = 0; b < n_tables; ++b) {
        double U = c0 * tables[b]->dt_max;
        g->dt_max[b] = tables[b]->dt_max;
        hb[b].U = U;
        hb[b].h = (float)(grid->h / U);
        for (int a = 0; a < 3; ++a) hb[b].org[a] = (float)(grid->origin[a] / U);
        // Is Phi just below the cut-off non-negligible? (table: its sample at dt_max)
        std::vector<double> phi;
        if (phi_kind == PHI_TABLE) {
            phi.resize(tables[b]->n);
            cudaError_t ce = cudaMemcpy(phi.data(), tables[b]->d_phi, sizeof(double) * phi.size(), cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) {
                rc = cuda_fail(ce, "fft_geom_create: table copy");
                free_geom(g);
                return rc;
            }
        } else {   // the series on 4096 points of [0, dt_max]
            phi.resize(4096);
            for (size_t k = 0; k < phi.size(); ++k) {
                const double dt = tables[b]->dt_max * (double)k / (double)(phi.size() - 1);
                double acc = 0.0;
                for (int j = 1; j <= tables[b]->n; ++j) acc += tables[b]->coef[j - 1] * sin(j * tables[b]->dw * dt);
                phi[k] = acc;
            }
        }
        double mx = 0.0;
        for (double v : phi) mx = fmax(mx, fabs(v));
        hb[b].sharp = (fabs(phi[phi.size() - 1]) > 1e-7 * mx) ? 1 : 0;
        hb[b].pad = 0;
        g->band[b] = hb[b];
    }
    bool any_sharp = false;
    for (int b = 0; b < n_tables; ++b) any_sharp = any_sharp || hb[b].sharp;
    g->sharp = any_sharp && dt_mode != FFT_DT_FP64;
    const bool need64 = (dt_mode == FFT_DT_FP64) || any_sharp;
    GEOM_TRY(dmalloc(g, &g->d_band, n_tables));
    GEOM_CUDA(cudaMemcpy(g->d_band, hb.data(), sizeof(BandConst) * n_tables, cudaMemcpyHostToDevice));

    // ---- tables in the device layout
    GEOM_TRY(dmalloc(g, &g->tab, (size_t)n_tables * g->n_tab));
    if (phi_kind == PHI_TABLE) {
        for (int b = 0; b < n_tables; ++b) {
            pack_table_kernel<<<(unsigned)ceil_div(g->n_tab, 256), 256>>>(tables[b]->d_phi, g->n_tab,
                                                                            g->tab + (size_t)b * g->n_tab);
            GEOM_CUDA(cudaGetLastError());
        }
    } else {
        // per band: (theta, 0), (0, 0), then a_1 .. a_{4 nq} as float pairs (zeros past n)
        std::vector<float2> packed((size_t)n_tables * n_tab, make_float2(0.0f, 0.0f));
        for (int b = 0; b < n_tables; ++b) {
            float2* blk = packed.data() + (size_t)b * n_tab;
            blk[0].x = (float)(tables[b]->dw * tables[b]->dt_max);
            float* a = reinterpret_cast<float*>(blk + 2);
            for (int j = 0; j < tables[b]->n; ++j) a[j] = (float)tables[b]->coef[j];
        }
        GEOM_CUDA(cudaMemcpy(g->tab, packed.data(), sizeof(float2) * packed.size(), cudaMemcpyHostToDevice));
    }

    // ---- row records
    {
        std::vector<RowRec> rec(n_rows);
        std::vector<RowRec64> rec64(need64 ? n_rows : 0);
        std::vector<int32_t> rb(n_rows);
        const double h3 = grid->h * grid->h * grid->h;
        for (int64_t p = 0; p < n_rows; ++p) {
            const double* xs = tx_xyz + 3 * rows[2 * p];
            const double* xr = tx_xyz + 3 * rows[2 * p + 1];
            int b = band_of_row ? band_of_row[p] : 0;
            rb[p] = b;
            double U = hb[b].U;
            double ax = xr[0] - xs[0], ay = xr[1] - xs[1], az = xr[2] - xs[2];
            double L = sqrt(ax * ax + ay * ay + az * az);
            if (!(L > 0)) {
                free_geom(g);
                set_error("fft_geom_create: a row has coincident emitter and receiver positions");
                return FFT_ERR_ARG;
            }
            RowRec& R = rec[p];
            R.a = make_float4((float)(0.5 * (xs[0] + xr[0]) / U), (float)(0.5 * (xs[1] + xr[1]) / U),
                              (float)(0.5 * (xs[2] + xr[2]) / U), (float)(0.5 * L / U));
            // K0 dV = -L h^3 / (2 pi c0^3 R_xs R_xr) Phi = C Phi / (Rs_band Rr_band)
            double C = -L * h3 / (2.0 * M_PI * c0 * c0 * c0 * U * U);
            R.b = make_float4((float)(ax / L), (float)(ay / L), (float)(az / L), (float)C);
            if (need64) {
                for (int a = 0; a < 3; ++a) {
                    rec64[p].xs[a] = xs[a];
                    rec64[p].xr[a] = xr[a];
                }
            }
        }
        GEOM_TRY(dmalloc(g, &g->rec, n_rows));
        GEOM_TRY(dmalloc(g, &g->row_band, n_rows));
        GEOM_CUDA(cudaMemcpy(g->rec, rec.data(), sizeof(RowRec) * n_rows, cudaMemcpyHostToDevice));
        GEOM_CUDA(cudaMemcpy(g->row_band, rb.data(), sizeof(int32_t) * n_rows, cudaMemcpyHostToDevice));
        if (need64) {
            GEOM_TRY(dmalloc(g, &g->rec64, n_rows));
            GEOM_CUDA(cudaMemcpy(g->rec64, rec64.data(), sizeof(RowRec64) * n_rows, cudaMemcpyHostToDevice));
        }
    }

    // ---- tiles
    g->tiles[0] = (int32_t)ceil_div(grid->nx, TILE_X);
    g->tiles[1] = (int32_t)ceil_div(grid->ny, TILE_Y);
    g->tiles[2] = (int32_t)ceil_div(grid->nz, TILE_Z);
    g->n_tiles = (int64_t)g->tiles[0] * g->tiles[1] * g->tiles[2];
    if (g->n_tiles >= (int64_t)INT32_MAX) {
        free_geom(g);
        set_error("fft_geom_create: grid too large");
        return FFT_ERR_ARG;
    }

    // Guarded kernels are needed only if a voxel centre of the tile-padded lattice coincides
    // (to within 1e-3 h) with a transducer: there R_xs = 0 and the plain form divides 0 by 0.
    for (int t = 0; t < n_tx && !g->guard; ++t) {
        bool on = true;
        for (int a = 0; a < 3; ++a) {
            double u = (tx_xyz[3 * t + a] - grid->origin[a]) / grid->h;
            double ru = nearbyint(u);
            int lim = g->tiles[a] * (a == 0 ? TILE_X : (a == 1 ? TILE_Y : TILE_Z));
            if (fabs(u - ru) > 1e-3 || ru < 0 || ru >= lim) on = false;
        }
        if (on) g->guard = true;
    }

    CullParams C;
    C.rec = g->rec;
    C.row_band = g->row_band;
    C.bc = g->d_band;
    C.M = n_rows;
    C.tiles_x = g->tiles[0];
    C.nx = grid->nx;
    C.ny = grid->ny;
    C.nz = grid->nz;
    C.tiles_y = g->tiles[1];

    std::vector<int64_t> tcnt(g->n_tiles), toff(g->n_tiles + 1, 0);
    // sharp geometries keep each tile's plain rows ahead of its sharp-band rows, so that the
    // two kinds run in separate launches (the plain kernels need fewer registers)
    const bool split = g->sharp;
    int64_t* d_nplain = nullptr;
    {
        int64_t* d_cnt = nullptr;
        GEOM_TRY(dmalloc(g, &g->tile_off, g->n_tiles + 1));
        d_cnt = g->tile_off;   // counts first, offsets after
        if (split) GEOM_CUDA(cudaMalloc(&d_nplain, sizeof(int64_t) * g->n_tiles));
        tile_count_kernel<<<(unsigned)g->n_tiles, CULL_THREADS>>>(C, split ? 1 : 0, d_cnt, d_nplain);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpy(tcnt.data(), d_cnt, sizeof(int64_t) * g->n_tiles, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && split) {
            g->tile_nplain.resize(g->n_tiles);
            e = cudaMemcpy(g->tile_nplain.data(), d_nplain, sizeof(int64_t) * g->n_tiles, cudaMemcpyDeviceToHost);
        }
        for (int64_t T = 0; T < g->n_tiles; ++T) toff[T + 1] = toff[T] + tcnt[T];
        g->E = toff[g->n_tiles];
        if (e == cudaSuccess)
            e = cudaMemcpy(g->tile_off, toff.data(), sizeof(int64_t) * (g->n_tiles + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) cudaFree(d_nplain);
        GEOM_CUDA(e);
    }
    {
        fft_status r2 = dmalloc(g, &g->tile_rows, g->E);
        if (r2 == FFT_OK && g->E > 0) {
            tile_fill_kernel<<<(unsigned)g->n_tiles, CULL_THREADS>>>(C, g->tile_off, d_nplain, g->tile_rows);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) r2 = cuda_fail(e, "tile lists");
        }
        cudaFree(d_nplain);
        GEOM_TRY(r2);
    }

    // ---- FP64 pair-frame bases of the entries
    GEOM_TRY(dmalloc(g, &g->ebase, g->E));
    GEOM_TRY(dmalloc(g, &g->ebase3, g->E));
    if (g->E > 0) {
        double* d_tx = nullptr;
        int32_t* d_pairs = nullptr;
        cudaError_t e = cudaMalloc(&d_tx, sizeof(double) * 3 * n_tx);
        if (e == cudaSuccess) e = cudaMalloc(&d_pairs, sizeof(int32_t) * 2 * n_rows);
        if (e == cudaSuccess) e = cudaMemcpy(d_tx, tx_xyz, sizeof(double) * 3 * n_tx, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_pairs, rows, sizeof(int32_t) * 2 * n_rows, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            entry_base_kernel<<<(unsigned)g->n_tiles, 256>>>(g->tile_off, g->tile_rows, d_tx, d_pairs, g->row_band,
                                                             g->d_band, grid->origin[0], grid->origin[1],
                                                             grid->origin[2], grid->h, g->tiles[0], g->tiles[1],
                                                             g->ebase, g->ebase3);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(d_tx);
        cudaFree(d_pairs);
        GEOM_CUDA(e);
    }

    // ---- row-major view of the entries
    {
        int32_t* d_rc = nullptr;
        int32_t* d_cur = nullptr;
        cudaError_t ea = cudaMalloc(&d_rc, sizeof(int32_t) * n_rows);
        if (ea == cudaSuccess) ea = cudaMalloc(&d_cur, sizeof(int32_t) * n_rows);
        if (ea == cudaSuccess) ea = cudaMemset(d_rc, 0, sizeof(int32_t) * n_rows);
        if (ea == cudaSuccess) ea = cudaMemset(d_cur, 0, sizeof(int32_t) * n_rows);
        if (ea != cudaSuccess) {
            cudaFree(d_rc);
            cudaFree(d_cur);
        }
        GEOM_CUDA(ea);
        if (g->E > 0) row_count_kernel<<<(unsigned)ceil_div(g->E, 256), 256>>>(g->tile_rows, g->E, d_rc);
        std::vector<int32_t> rc32(n_rows);
        cudaError_t e = cudaMemcpy(rc32.data(), d_rc, sizeof(int32_t) * n_rows, cudaMemcpyDeviceToHost);
        std::vector<int64_t> roff(n_rows + 1, 0);
        for (int64_t p = 0; p < n_rows; ++p) roff[p + 1] = roff[p] + rc32[p];
        fft_status r2 = (e == cudaSuccess) ? dmalloc(g, &g->row_off, n_rows + 1) : cuda_fail(e, "row counts");
        if (r2 == FFT_OK) r2 = dmalloc(g, &g->row_ent, g->E);
        if (r2 == FFT_OK) {
            e = cudaMemcpy(g->row_off, roff.data(), sizeof(int64_t) * (n_rows + 1), cudaMemcpyHostToDevice);
            if (e == cudaSuccess && g->E > 0) {
                row_fill_kernel<<<(unsigned)ceil_div(g->E, 256), 256>>>(g->tile_rows, g->E, g->row_off, d_cur,
                                                                        g->row_ent);
                row_sort_kernel<<<(unsigned)ceil_div(n_rows, 128), 128>>>(g->row_off, n_rows, g->row_ent);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) r2 = cuda_fail(e, "row lists");
        }
        cudaFree(d_rc);
        cudaFree(d_cur);
        GEOM_TRY(r2);
    }

    // ---- work items
    GEOM_TRY(set_apply_attributes(g));
    // commit the no-allocation PSF's static scratch on this device now, so that
    // fft_psf_noalloc itself never loads a module or allocates
    GEOM_TRY(noalloc_prepare(g->dev));
    g->apply_ctas = apply_occupancy(g);
    sharp_launch_shape(g);
    plain_launch_shape(g);
    GEOM_TRY(dmalloc(g, &g->jpart, (size_t)g->E * 4));   // one J partial per (entry, 8 x 8 x 8 region)
    GEOM_TRY(dmalloc(g, &g->counter, 4));
    GEOM_TRY(build_items(g, toff, DEFAULT_ITEMS_PER_CTA));
    GEOM_CUDA(cudaDeviceSynchronize());
    GEOM_TRY(count_support(g, &g->support, &g->evaluated));
    GEOM_CUDA(cudaDeviceSynchronize());
#undef GEOM_TRY
#undef GEOM_CUDA
    *out = g;
    return FFT_OK;
}

extern "C" void fft_geom_destroy(fft_geom g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->dev) cudaSetDevice(g->dev);
    cudaDeviceSynchronize();
    int dev = g->dev;
    free_geom(g);
    if (cur != dev) cudaSetDevice(cur);
}

extern "C" fft_status fft_geom_info(fft_geom g, fft_geom_info_t* info) {
    FFT_ARG(g && info, "fft_geom_info: null argument");
    info->n_rows = g->M;
    info->n_vox = g->V;
    info->n_entries = g->E;
    info->n_items = g->n_items;
    info->support_evals = g->support;
    info->evaluated_evals = g->evaluated;
    info->scratch_bytes = g->scratch_bytes;
    info->dt_mode = g->dt_mode;
    info->phi_terms = g->trig_terms;
    info->psf_tc_mma_flops = g->psf_tc_mma_flops;
    info->psf_tc_entries = g->psf_tc_entries;
    return FFT_OK;
}
