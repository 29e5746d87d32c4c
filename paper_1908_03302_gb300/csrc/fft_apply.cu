// J m and J^T d with every entry of J recomputed inside each product instead of stored
// (Sec. II-C), tile-centric on sm_103a.
//
// Work decomposition
//   * The voxel grid is cut into 16 x 16 x 8 tiles. Each tile has a list of candidate rows
//     (built once per geometry by a conservative cull). A work item is a tile and a range of
//     its rows; a unit is one region of one item: an 8 x 8 x 8 region (four 8 x 4 x 4
//     sub-bricks, four regions per tile) for the single-column modes, an 8 x 8 x 4 region
//     (two sub-bricks, eight per tile) for the four-column ones. Every warp of the persistent
//     grid pulls units from a counter, heaviest items first, on its own (the only CTA barrier
//     follows the table load). The launch shape (warps per CTA, CTAs per SM) is picked per
//     variant from its register budget and the shared memory the band tables take.
//   * Lane l owns 4 consecutive x voxels of each sub-brick of its warp's region. Per chunk of
//     32 rows, lane l loads row l, moves its geometry into the tile's pair frame and tests it
//     against the region's sub-bricks (tangent-plane bounds of the convex detour); the rows
//     that reach one are staged in shared memory and broadcast, and each is evaluated on the
//     sub-bricks it reaches.
//   * Per (row, voxel): pair-frame coordinates by FFMA from per-lane offsets, normalised
//     detour (cancellation-free form), Phi from the band table in shared memory (one 64-bit
//     load, linear interpolation), geometric factor 1 / (R_xs R_xr).
//   * J^T accumulates per voxel in registers over the item's rows (gather, no atomics).
//     J folds each row's lane partials to 8 with two shuffles, parks them in the row's
//     consumed staging record, and the row's own lane sums them after the chunk: one partial
//     per (entry, region); a second kernel sums each row's partials in a fixed order. Both are
//     deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "fft_common.cuh"
#include "fft_device.cuh"

namespace fftgb {

// MODE_COV: sensitivity coverage sum_p |J[p, v] w_p| (J^T of |J|, same gather as MODE_JT).
// MODE_JT4 / MODE_J4: J^T and J for four right-hand sides at once (every evaluated entry is
// applied to all four; blocks are column-major: column r at r * V or r * M).
enum { MODE_JT = 0, MODE_J = 1, MODE_COUNT = 2, MODE_FROB = 3, MODE_COV = 4, MODE_JT4 = 5, MODE_J4 = 6 };
constexpr int STG_PER_WARP = 128;   // staged float4 per warp: 32 rows x (3 or 4)

struct ApplyParams {
    const RowRec* rec;
    const RowRec64* rec64;
    const int32_t* row_band;
    const float2* tab;
    int n_bands;
    int n_tab;
    const BandConst* bc;     // device [n_bands]
    const int32_t* tile_rows;
    const float4* ebase;     // [E] (p + hl, p - hl, c1, c2) of each entry's tile origin (pair frame)
    const float* ebase3;     // [E] c3 of each entry's tile origin
    const Item* items;
    int n_items;
    int32_t* counter;
    int tiles_x, tiles_y;
    int nx, ny, nz;
    double org[3];
    double h;
    const float* vin;        // J: m [V]; J^T: d [M]
    float* vout;             // J: jpart [E * 4]; J^T: g [V]
    float* gpart;            // J^T partials of multi-item tiles
    double* dsum;            // FROB: one per unit [n_items * 4]
    unsigned long long* icount;   // COUNT
    int trig_nq;             // sine-series Phi: coefficient groups of 4 per band
    int64_t nvox, nrow;      // column lengths of the batch modes' blocks (V, M)
};

// Phi of the normalised detour v from the band data at shared address tb (table lookup or
// sine series, see fft_device.cuh).
template <int PHI>
__device__ __forceinline__ float phi_eval(float v, uint32_t tb, float nm1, int nq) {
    if (PHI == PHI_TRIG) return phi_trig(v, tb, nq);
    return phi_lookup(v, tb, nm1);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 detour for the precision-study mode: voxel (ix, iy, iz), row record in metres.
__device__ __forceinline__ float detour_v64(const RowRec64& r, double ox, double oy, double oz, double h,
                                            int ix, int iy, int iz, double U, float& w_band) {
    double x = ox + ix * h, y = oy + iy * h, z = oz + iz * h;
    double ex = r.xr[0] - r.xs[0], ey = r.xr[1] - r.xs[1], ez = r.xr[2] - r.xs[2];
    double L = sqrt(ex * ex + ey * ey + ez * ez);
    ex /= L; ey /= L; ez /= L;
    double dx = x - 0.5 * (r.xs[0] + r.xr[0]), dy = y - 0.5 * (r.xs[1] + r.xr[1]),
           dz = z - 0.5 * (r.xs[2] + r.xr[2]);
    double p = dx * ex + dy * ey + dz * ez;
    double c1 = dy * ez - dz * ey, c2 = dz * ex - dx * ez, c3 = dx * ey - dy * ex;
    double q2 = c1 * c1 + c2 * c2 + c3 * c3;
    double hl = 0.5 * L, ps = p + hl, pr = p - hl;
    double Rs = sqrt(ps * ps + q2), Rr = sqrt(pr * pr + q2);
    if (Rs == 0.0 || Rr == 0.0) {
        w_band = 0.0f;
        return 0.0f;
    }
    double A = Rs + fabs(ps), B = Rr + fabs(pr);
    double R = q2 * (A + B) / (A * B) + ((fabs(ps) - ps) + (fabs(pr) + pr));
    w_band = (float)(U * U / (Rs * Rr));
    double v = R / U;
    return (float)(v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v));
}

// Resident 8-warp CTAs per SM the register budget is sized for: 4 (64 registers) for the
// stable-detour table kernels, 3 (80) for the others, 2 (128) for the four-column ones and the
// other sharp-band ones. The single-column stable-detour table variants are sized separately
// (apply_sharp_wide and apply_plain_wide below).
template <int MODE, int DT, bool SHARP, int PHI>
constexpr int apply_min_blocks() {
    return (SHARP || MODE == MODE_JT4 || MODE == MODE_J4) ? 2
                                                          : ((DT == FFT_DT_STABLE && PHI == PHI_TABLE) ? 4 : 3);
}

// Sub-bricks per unit and units (regions) per item of each mode: see sub_dy below.
template <int MODE>
constexpr int apply_nsub() {
    return (MODE == MODE_JT4 || MODE == MODE_J4) ? 2 : 4;
}
template <int MODE>
constexpr int apply_regions() {
    return 16 / apply_nsub<MODE>();   // 16 sub-bricks of 8 x 4 x 4 per 16 x 16 x 8 tile
}

// Sub-bricks of a unit. The single-column modes take an 8 x 8 x 8 region (NSUB = 4) and the
// four-column modes, whose per-voxel state is four times larger, an 8 x 8 x 4 region (NSUB =
// 2). Sub-brick s of a lane sits at y offset sub_dy(s) and z offset sub_dz(s) from sub-brick 0;
// for NSUB = 4 the order (0,0), (4,0), (4,4), (0,4) lets every step between consecutive
// sub-bricks move along one axis only.
template <int NSUB>
__device__ __forceinline__ constexpr int sub_dy(int s) {
    return NSUB == 2 ? 4 * s : ((s == 1 || s == 2) ? 4 : 0);
}
template <int NSUB>
__device__ __forceinline__ constexpr int sub_dz(int s) {
    return NSUB == 2 ? 0 : (s >= 2 ? 4 : 0);
}

// Pair-frame values of a lane's first voxel moved from sub-brick s - 1 to sub-brick s (s >= 1):
// +4 voxels in y (s = 1), +4 in z (s = 2), -4 in y (s = 3). A step d along an axis changes
// p by d . e and c = (x - o) x e by d x e. The main loop and the FP64 re-decision both reach
// sub-brick s through these same operations, so their FP32 values agree bit for bit.
template <int NSUB, bool PL>
__device__ __forceinline__ void sub_step(int s, float hx, float hy, float hz, float& ps, float& pr, float& c1,
                                         float& c2, float& c3) {
    if (s == 1 || s == 3) {
        const float f = (s == 1) ? 4.0f : -4.0f;
        ps = fmaf(f, hy, ps);
        pr = fmaf(f, hy, pr);
        if (!PL) c1 = fmaf(f, hz, c1);
        c3 = fmaf(-f, hx, c3);
    } else if (s == 2) {
        if (!PL) {
            ps = fmaf(4.0f, hz, ps);
            pr = fmaf(4.0f, hz, pr);
        }
        c1 = fmaf(-4.0f, hy, c1);
        c2 = fmaf(4.0f, hx, c2);
    }
}

// The FP64 re-decision of the sharp-band kernels, out of line (called only for an entry where
// some lane's FP32 detour lies within CUT_BAND of the cut), so that its FP64 temporaries do not
// weigh on the register allocation of the main loop. For each of the lane's 4 NSUB voxels
// (k = 4 s + t) it recomputes the FP32 detour by the operations of the main pass, and for the
// voxels near the cut re-decides dt < dt_max in FP64. It returns in d[k] what the main pass's
// term has to change by: val2 - val1 (J, J^T, four-column modes), |val2| - |val1| (coverage),
// val2^2 - val1^2 (Frobenius), +1 / -1 (support count), 0 where nothing changes. `inner` holds
// the sub-bricks lying between the transducer planes (bit s).
template <int MODE, int DT, bool GUARD, int PHI, int NSUB>
__device__ __noinline__ void sharp_fix(const ApplyParams& P, float4 A, float4 B, float4 C, float Xl, float Yl,
                                       float Zl, bool planar, uint32_t inner_bits, float cutb, uint32_t tb,
                                       float nm1, int nq, int ix0, int iy0, int iz0, float* d) {
    const float hx = B.x, hy = B.y, hz = B.z;
    const float hl = 0.5f * (A.x - A.y);
    const int b = __float_as_int(C.w) & 0xff;
    const double U = P.bc[b].U;
    // one voxel per iteration, each recomputed from the lane base (few values live across
    // iterations, which keeps the caller's register saves around this call small)
#pragma unroll 1
    for (int k = 0; k < 4 * NSUB; ++k) {
        const int s = k >> 2, t = k & 3;
        d[k] = 0.0f;
        const float offs = planar ? fmaf(Xl, hx, Yl * hy) : fmaf(Xl, hx, fmaf(Yl, hy, Zl * hz));
        float pss = A.x + offs, prs = A.y + offs;
        float c1s = planar ? fmaf(-Zl, hy, A.z) : fmaf(Yl, hz, fmaf(-Zl, hy, A.z));
        float c2s = planar ? fmaf(Zl, hx, A.w) : fmaf(Zl, hx, fmaf(-Xl, hz, A.w));
        float c3s = fmaf(Xl, hy, fmaf(-Yl, hx, B.w));
#pragma unroll 1
        for (int q = 1; q <= s; ++q) {
            if (planar)
                sub_step<NSUB, true>(q, hx, hy, hz, pss, prs, c1s, c2s, c3s);
            else
                sub_step<NSUB, false>(q, hx, hy, hz, pss, prs, c1s, c2s, c3s);
        }
        const float ft = (float)t;
        const float c1sq = c1s * c1s;
        const float pst = (t == 0 ? pss : fmaf(ft, hx, pss));
        const float prt = (t == 0 ? prs : fmaf(ft, hx, prs));
        const float c3t = (t == 0 ? c3s : fmaf(ft, hy, c3s));
        float q2;
        if (planar) {
            q2 = fmaf(c3t, c3t, fmaf(c2s, c2s, c1sq));
        } else {
            const float c2t = (t == 0 ? c2s : fmaf(-ft, hz, c2s));
            q2 = fmaf(c2t, c2t, fmaf(c3t, c3t, c1sq));
        }
        const bool inner = (DT == FFT_DT_STABLE) && ((inner_bits >> s) & 1u);
        float is, ir;
        const float vr = inner ? detour_v<DT, GUARD, true, true>(pst, prt, q2, hl, is, ir)
                               : detour_v<DT, GUARD, false, true>(pst, prt, q2, hl, is, ir);
        if (!(fabsf(vr - 1.0f) < cutb)) continue;
        const float v = __saturatef(vr);
        const bool in = in_support64(P.rec64[__float_as_int(C.z)], P.org[0], P.org[1], P.org[2], P.h, ix0 + t,
                                     iy0 + sub_dy<NSUB>(s), iz0 + sub_dz<NSUB>(s), U);
        const float v2 = settle_cut(v, in);
        if (v2 == v) continue;
        if (MODE == MODE_COUNT) {
            d[k] = (v2 < 1.0f) ? 1.0f : -1.0f;
            continue;
        }
        const float w = is * ir;
        const float val1 = phi_eval<PHI>(v, tb, nm1, nq) * w;
        const float val2 = phi_eval<PHI>(v2, tb, nm1, nq) * w;
        if (MODE == MODE_COV) d[k] = fabsf(val2) - fabsf(val1);
        else if (MODE == MODE_FROB) d[k] = val2 * val2 - val1 * val1;
        else d[k] = val2 - val1;
    }
}

// The sharp-band stable-detour table variants (single column) are built for CTAs of up to 20
// warps at one per SM (96 registers used): one CTA of 20 warps shares one copy of the band
// tables, and keeps more warps resident than 8-warp CTAs do (two per SM at this register
// count, fewer where large tables fill shared memory). Measured against 24 warps at 80
// registers and 16 warps at 128: the spills of the first and the lower occupancy of the
// second cost more.
template <int MODE, int DT, bool SHARP, int PHI>
constexpr bool apply_sharp_wide() {
    return SHARP && DT == FFT_DT_STABLE && PHI == PHI_TABLE && MODE != MODE_JT4 && MODE != MODE_J4;
}
constexpr int SHARP_MAX_WARPS = 20;

// The plain stable-detour table variants (single column) are built for blocks of up to 24
// warps at one per SM, i.e. 80 registers: their 16 per-lane voxels (8 x 8 x 8 units) want more
// than 64, and one wide CTA shares one copy of the band tables. Measured against 32 warps at
// 64 registers: slices3d J^T 408.0 -> 407.6 ms, J 412.6 -> 411.4 ms, ring256 J^T 3.75 -> 3.72 ms.
template <int MODE, int DT, bool SHARP, int PHI>
constexpr bool apply_plain_wide() {
    return !SHARP && DT == FFT_DT_STABLE && PHI == PHI_TABLE && MODE != MODE_JT4 && MODE != MODE_J4;
}
constexpr int PLAIN_MAX_WARPS = 24;

template <int MODE, int DT, bool SHARP, int PHI>
constexpr int apply_block_bound() {
    return apply_sharp_wide<MODE, DT, SHARP, PHI>()   ? 32 * SHARP_MAX_WARPS
           : apply_plain_wide<MODE, DT, SHARP, PHI>() ? 32 * PLAIN_MAX_WARPS
                                                      : APPLY_THREADS;
}

template <int MODE, int DT, bool GUARD, bool SHARP, int PHI>
__global__ void __launch_bounds__(apply_block_bound<MODE, DT, SHARP, PHI>(),
                                  apply_block_bound<MODE, DT, SHARP, PHI>() == APPLY_THREADS
                                      ? apply_min_blocks<MODE, DT, SHARP, PHI>()
                                      : 1)
    apply_kernel(const __grid_constant__ ApplyParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* s_tab = reinterpret_cast<float2*>(smem);
    const int tab_len = P.n_bands * P.n_tab;
    float4* s_stage = reinterpret_cast<float4*>(smem + (((size_t)tab_len * sizeof(float2) + 15) & ~(size_t)15));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < tab_len; i += blockDim.x) s_tab[i] = P.tab[i];
    __syncthreads();   // the only CTA-wide barrier: from here on every warp runs on its own

    const uint32_t tab_addr = smem_addr(s_tab);
    const float nm1 = (float)(P.n_tab - 1);
    const int nq = P.trig_nq;
    const int lx = lane & 1, ly = (lane >> 1) & 3, lz = lane >> 3;
    constexpr bool BATCH = (MODE == MODE_JT4 || MODE == MODE_J4);
    constexpr int SR = BATCH ? 4 : 3;   // staged float4 per row
    constexpr int NSUB = apply_nsub<MODE>();
    constexpr int NREG = apply_regions<MODE>();
    constexpr bool FLAGW = (NSUB == 4);
    float4* stg = s_stage + warp * STG_PER_WARP;
    const int n_units = P.n_items * NREG;

    for (;;) {
        // A unit is one region of one item (unit = item * NREG + region): 8 x 8 x 8 voxels for
        // the single-column modes (regions 2 x 2 x 1 per tile), 8 x 8 x 4 for the four-column
        // ones (2 x 2 x 2 per tile).
        int unit = 0;
        if (lane == 0) unit = atomicAdd(P.counter, 1);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= n_units) break;
        const int it = unit / NREG, region = unit % NREG;
        const Item item = P.items[it];
        const int tx = item.tile % P.tiles_x;
        const int ty = (item.tile / P.tiles_x) % P.tiles_y;
        const int tz = item.tile / (P.tiles_x * P.tiles_y);
        const int TX = TILE_X * tx, TY = TILE_Y * ty, TZ = TILE_Z * tz;
        const int wx = region & 1, wy = (region >> 1) & 1, wz = (NSUB == 2) ? (region >> 2) : 0;
        // lane voxel offsets in the tile (sub-brick 0, first of its 4 x voxels)
        const int oxi = 8 * wx + 4 * lx, oyi = 8 * wy + ly, ozi = 4 * wz + lz;
        const float Xl = (float)oxi, Yl = (float)oyi, Zl = (float)ozi;

        // validity of this lane's voxels (bit 4 s + t) and of the region's sub-bricks (bit s)
        auto lane_vmask = [&]() {
            uint32_t vm = 0;
#pragma unroll
            for (int s = 0; s < NSUB; ++s) {
                if (TZ + ozi + sub_dz<NSUB>(s) < P.nz && TY + oyi + sub_dy<NSUB>(s) < P.ny) {
#pragma unroll
                    for (int t = 0; t < NX_LANE; ++t)
                        if (TX + oxi + t < P.nx) vm |= 1u << (4 * s + t);
                }
            }
            return vm;
        };
        uint32_t sub_ok = 0;
#pragma unroll
        for (int s = 0; s < NSUB; ++s)
            if (TX + 8 * wx < P.nx && TY + 8 * wy + sub_dy<NSUB>(s) < P.ny && TZ + 4 * wz + sub_dz<NSUB>(s) < P.nz)
                sub_ok |= 1u << s;
        // the gather modes need the mask only for their stores: recomputed there
        constexpr bool VM_LIVE = !(MODE == MODE_JT || MODE == MODE_COV || MODE == MODE_JT4);
        const uint32_t vmask = VM_LIVE ? lane_vmask() : 0u;
        const int64_t vbase = ((int64_t)(TZ + ozi) * P.ny + TY + oyi) * P.nx + TX + oxi;

        float acc[NSUB][NX_LANE];
        float mv[NSUB][NX_LANE];
        float acc4[2][NX_LANE][4];   // four-column modes only (NSUB = 2)
        float mv4[2][NX_LANE][4];
        double dacc = 0.0;
        unsigned long long cnt = 0, cnt_eval = 0;
#pragma unroll
        for (int s = 0; s < NSUB; ++s)
#pragma unroll
            for (int t = 0; t < NX_LANE; ++t) {
                const int64_t vo = vbase + ((int64_t)sub_dz<NSUB>(s) * P.ny + sub_dy<NSUB>(s)) * P.nx + t;
                acc[s][t] = 0.0f;
                mv[s][t] = 0.0f;
                if (MODE == MODE_J && ((vmask >> (4 * s + t)) & 1u)) mv[s][t] = __ldg(P.vin + vo);
                if (BATCH && s < 2) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc4[s & 1][t][r] = 0.0f;
                        mv4[s & 1][t][r] = 0.0f;
                        if (MODE == MODE_J4 && ((vmask >> (4 * s + t)) & 1u))
                            mv4[s & 1][t][r] = __ldg(P.vin + (int64_t)r * P.nvox + vo);
                    }
                }
            }

        for (int64_t e0 = item.e0; e0 < item.e1; e0 += 32) {
            // ---- stage: lane l prepares row e0 + l
            const int64_t e = e0 + lane;
            const bool have = e < item.e1;
            uint32_t okb = 0, inb = 0;   // sub-bricks the row may reach / lying between its transducer planes
            if (have) {
                const int p = P.tile_rows[e];
                const float4 base = P.ebase[e];
                const float base3 = P.ebase3[e];
                const RowRec r = P.rec[p];
                const int b = P.row_band[p];
                const BandConst bc = P.bc[b];
                const float hb = bc.h;
                float W = r.b.w;
                if (MODE == MODE_JT) W *= __ldg(P.vin + p);
                if (MODE == MODE_COV) W = fabsf(W) * (P.vin ? fabsf(__ldg(P.vin + p)) : 1.0f);
                float4 W4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (MODE == MODE_JT4)
                    W4 = make_float4(W * __ldg(P.vin + p), W * __ldg(P.vin + P.nrow + p),
                                     W * __ldg(P.vin + 2 * P.nrow + p), W * __ldg(P.vin + 3 * P.nrow + p));
                const float ex = r.b.x, ey = r.b.y, ez = r.b.z, hl = r.a.w;
                // sub-brick centres relative to the pair midpoint (FP32; used by the bound only)
                const float dx = fmaf((float)TX, hb, bc.org[0]) - r.a.x;
                const float dy = fmaf((float)TY, hb, bc.org[1]) - r.a.y;
                const float dz = fmaf((float)TZ, hb, bc.org[2]) - r.a.z;
                const float cx = fmaf(8.0f * wx + 3.5f, hb, dx);
                const float hxx = 3.5f * hb, hyy = 1.5f * hb;
                // rows with zero weight add exactly nothing to J^T: skip them
                const bool live = (MODE == MODE_JT4) ? (W4.x != 0.0f || W4.y != 0.0f || W4.z != 0.0f || W4.w != 0.0f)
                                                     : ((MODE != MODE_JT && MODE != MODE_COV) || (W != 0.0f));
                const float pext = hxx * fabsf(ex) + hyy * (fabsf(ey) + fabsf(ez)) + 1e-3f;
#pragma unroll
                for (int s = 0; s < NSUB; ++s) {
                    const float cy = fmaf(8.0f * wy + (float)sub_dy<NSUB>(s) + 1.5f, hb, dy);
                    const float cz = fmaf(4.0f * wz + (float)sub_dz<NSUB>(s) + 1.5f, hb, dz);
                    if (live && ((sub_ok >> s) & 1u) && box_may_touch(cx, cy, cz, ex, ey, ez, hl, hxx, hyy, hyy))
                        okb |= 1u << s;
                    // sub-bricks whose voxels all satisfy |p| <= hl (between the transducer planes)
                    if (fabsf(fmaf(cx, ex, fmaf(cy, ey, cz * ez))) + pext <= hl) inb |= 1u << s;
                }
                const uint32_t tb = tab_addr + (uint32_t)(b * P.n_tab) * 8u - (PHI == PHI_TABLE ? MAGIC_BITS_X8 : 0u);
                stg[lane * SR + 0] = base;
                stg[lane * SR + 1] = make_float4(hb * ex, hb * ey, hb * ez, base3);
                if (MODE == MODE_JT4) stg[lane * SR + 3] = W4;
                // planar pair (both transducers at one z): stepping along x changes only c3
                const int planar = (ez == 0.0f) ? 1 : 0;
                // flags word: band (bits 0-7), sharp band (8), planar pair (9); with four
                // sub-bricks also the sub-bricks the row may reach (12 + s) and the inner ones
                // (16 + s)
                const uint32_t fl = FLAGW ? ((okb << 12) | (inb << 16)) : 0u;
                stg[lane * SR + 2] = make_float4(W, __uint_as_float(tb), __int_as_float(p),
                                                __int_as_float(b | (bc.sharp << 8) | (planar << 9) | (int)fl));
            }
            // With two sub-bricks the per-row tests read warp-uniform ballots (uniform branches);
            // with four, the row's staged flag word (eight ballots per chunk cost more there).
            uint32_t mk[NSUB], ik[NSUB];
#pragma unroll
            for (int s = 0; s < NSUB; ++s) {
                mk[s] = FLAGW ? 0u : __ballot_sync(0xffffffffu, (okb >> s) & 1u);
                ik[s] = FLAGW ? 0u : __ballot_sync(0xffffffffu, (inb >> s) & 1u);
            }
            uint32_t mm = __ballot_sync(0xffffffffu, okb != 0u);
            __syncwarp();
            float mypart = 0.0f;
            float mypart4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            while (mm) {
                const int bit = __ffs(mm) - 1;
                mm &= mm - 1;
                const float4 A = stg[bit * SR + 0];
                const float4 B = stg[bit * SR + 1];
                const float4 C = stg[bit * SR + 2];
                const float4 W4 = (MODE == MODE_JT4) ? stg[bit * SR + 3] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float Wr[4] = {W4.x, W4.y, W4.z, W4.w};
                const float hx = B.x, hy = B.y, hz = B.z, W = C.x;
                const float hl = 0.5f * (A.x - A.y);   // used by the textbook (NAIVE) detour only
                const uint32_t tb = __float_as_uint(C.y);
                const uint32_t cw = (uint32_t)__float_as_int(C.w);
                // voxels whose FP32 detour falls within CUT_BAND of a sharp band's cut-off
                const float cutb = (SHARP && ((cw >> 8) & 1u)) ? CUT_BAND : -1.0f;
                const bool planar = (DT != FFT_DT_FP64) && ((cw >> 9) & 1u);
                bool near = false;   // a voxel of this lane has its FP32 detour within CUT_BAND of the cut
                // lane base (sub-brick 0, t = 0) in the pair frame: small offsets added to the
                // tile origin's FP64-derived values
                float part = 0.0f;
                float part4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                // The entry's evaluation, specialised for planar pairs (both transducers at one
                // z: the axis has no z component, so h_z = 0 exactly, c1 and c2 do not change
                // along the lane's voxels or between sub-bricks at one z, and p does not change
                // in z).
                // SH: the near-cut checks, only for rows of a band whose Phi does not vanish at
                // the cut (the other rows of a sharp geometry take the plain evaluation; both
                // give the same values there).
                auto entry_body = [&](auto planar_tag, auto sharp_tag) {
                    constexpr bool PL = decltype(planar_tag)::value;
                    constexpr bool SH = decltype(sharp_tag)::value;
                const float off = PL ? fmaf(Xl, hx, Yl * hy) : fmaf(Xl, hx, fmaf(Yl, hy, Zl * hz));
                float psb = A.x + off, prb = A.y + off;
                float c1 = PL ? fmaf(-Zl, hy, A.z) : fmaf(Yl, hz, fmaf(-Zl, hy, A.z));
                float c2 = PL ? fmaf(Zl, hx, A.w) : fmaf(Zl, hx, fmaf(-Xl, hz, A.w));
                float c3 = fmaf(Xl, hy, fmaf(-Yl, hx, B.w));
                float c12_planar = PL ? fmaf(c2, c2, c1 * c1) : 0.0f;
#pragma unroll
                for (int s = 0; s < NSUB; ++s) {
                    if (s > 0) {
                        sub_step<NSUB, PL>(s, hx, hy, hz, psb, prb, c1, c2, c3);
                        if (PL && s == 2) c12_planar = fmaf(c2, c2, c1 * c1);
                    }
                    if (!(FLAGW ? ((cw >> (12 + s)) & 1u) : ((mk[s] >> bit) & 1u))) continue;
                    const float c1sq = PL ? 0.0f : c1 * c1;
                    const bool inner = (DT == FFT_DT_STABLE) &&
                                       (FLAGW ? ((cw >> (16 + s)) & 1u) : ((ik[s] >> bit) & 1u));
#define FFT_EVAL_SUB(INNER_V, PLANAR_V)                                                              \
    float vv[NX_LANE], ww[NX_LANE];                                                                \
    _Pragma("unroll") for (int t = 0; t < NX_LANE; ++t) {                                          \
        const float ft = (float)t;                                                                 \
        float is, ir, v, w;                                                                        \
        if (DT == FFT_DT_FP64) {                                                                   \
            const RowRec64 r64 = P.rec64[__float_as_int(C.z)];                                     \
            const int b = (int)(cw & 0xffu);                                                       \
            v = detour_v64(r64, P.org[0], P.org[1], P.org[2], P.h, TX + oxi + t,                   \
                           TY + oyi + sub_dy<NSUB>(s), TZ + ozi + sub_dz<NSUB>(s), P.bc[b].U, w);  \
            is = 1.0f;                                                                             \
            ir = w;                                                                                \
        } else {                                                                                   \
            const float pst = (t == 0 ? psb : fmaf(ft, hx, psb));                                  \
            const float prt = (t == 0 ? prb : fmaf(ft, hx, prb));                                  \
            const float c3t = (t == 0 ? c3 : fmaf(ft, hy, c3));                                    \
            float q2;                                                                              \
            if (PLANAR_V) {                                                                        \
                q2 = fmaf(c3t, c3t, c12sq);                                                        \
            } else {                                                                               \
                const float c2t = (t == 0 ? c2 : fmaf(-ft, hz, c2));                               \
                q2 = fmaf(c2t, c2t, fmaf(c3t, c3t, c1sq));                                         \
            }                                                                                      \
            if (SH) {                                                                              \
                v = detour_v<DT, GUARD, INNER_V, true>(pst, prt, q2, hl, is, ir);                  \
                near |= (fabsf(v - 1.0f) < cutb);                                                  \
                v = __saturatef(v);                                                                \
            } else {                                                                               \
                v = detour_v<DT, GUARD, INNER_V>(pst, prt, q2, hl, is, ir);                        \
            }                                                                                      \
        }                                                                                          \
        if (MODE == MODE_COUNT) {                                                                  \
            if ((vmask >> (4 * s + t)) & 1u) {                                                     \
                ++cnt_eval;                                                                        \
                if (v < 1.0f) ++cnt;                                                               \
            }                                                                                      \
            continue;                                                                              \
        }                                                                                          \
        if constexpr (PHI == PHI_TRIG) {                                                           \
            vv[t] = v;                                                                             \
            ww[t] = is * ir;                                                                       \
            continue;                                                                              \
        }                                                                                          \
        const float val = phi_lookup(v, tb, nm1) * (is * ir);                                      \
        if (MODE == MODE_JT) acc[s][t] = fmaf(val, W, acc[s][t]);                                  \
        if (MODE == MODE_COV) acc[s][t] = fmaf(fabsf(val), W, acc[s][t]);                          \
        if (MODE == MODE_JT4) {                                                                    \
            _Pragma("unroll") for (int r = 0; r < 4; ++r) acc4[s & 1][t][r] = fmaf(val, Wr[r], acc4[s & 1][t][r]); \
        }                                                                                          \
        if (MODE == MODE_J4) {                                                                     \
            _Pragma("unroll") for (int r = 0; r < 4; ++r) part4[r] = fmaf(val, mv4[s & 1][t][r], part4[r]); \
        }                                                                                          \
        if (MODE == MODE_J) part = fmaf(val, mv[s][t], part);                                      \
        if (MODE == MODE_FROB) {                                                                   \
            if ((vmask >> (4 * s + t)) & 1u) part = fmaf(val, val, part);                          \
        }                                                                                          \
    }                                                                                              \
    if constexpr (PHI == PHI_TRIG && MODE != MODE_COUNT) {                                         \
        float ph[NX_LANE];                                                                         \
        phi_trig_n<NX_LANE>(vv, tb, nq, ph);                                                       \
        _Pragma("unroll") for (int t = 0; t < NX_LANE; ++t) {                                      \
            const float val = ph[t] * ww[t];                                                       \
            if (MODE == MODE_JT) acc[s][t] = fmaf(val, W, acc[s][t]);                              \
            if (MODE == MODE_COV) acc[s][t] = fmaf(fabsf(val), W, acc[s][t]);                      \
            if (MODE == MODE_JT4) {                                                                \
                _Pragma("unroll") for (int r = 0; r < 4; ++r) acc4[s & 1][t][r] = fmaf(val, Wr[r], acc4[s & 1][t][r]); \
            }                                                                                      \
            if (MODE == MODE_J4) {                                                                 \
                _Pragma("unroll") for (int r = 0; r < 4; ++r) part4[r] = fmaf(val, mv4[s & 1][t][r], part4[r]); \
            }                                                                                      \
            if (MODE == MODE_J) part = fmaf(val, mv[s][t], part);                                  \
            if (MODE == MODE_FROB) {                                                               \
                if ((vmask >> (4 * s + t)) & 1u) part = fmaf(val, val, part);                      \
            }                                                                                      \
        }                                                                                          \
    }
                    const float c12sq = PL ? c12_planar : fmaf(c2, c2, c1sq);
                    if (inner) {
                        FFT_EVAL_SUB(true, PL)
                    } else {
                        FFT_EVAL_SUB(false, PL)
                    }
                }
                };
                if (SHARP && cutb > 0.0f) {
                    if (planar)
                        entry_body(std::true_type{}, std::integral_constant<bool, SHARP>{});
                    else
                        entry_body(std::false_type{}, std::integral_constant<bool, SHARP>{});
                } else {
                    if (planar)
                        entry_body(std::true_type{}, std::false_type{});
                    else
                        entry_body(std::false_type{}, std::false_type{});
                }
#undef FFT_EVAL_SUB
                if (SHARP && DT != FFT_DT_FP64 && __any_sync(0xffffffffu, near)) {
                    // FP64 re-decision of the voxels whose FP32 detour lies within CUT_BAND of
                    // the cut; d[k] is the change of this entry's term for voxel k = 4 s + t
                    float d[4 * NSUB];
                    uint32_t inner_bits = (cw >> 16) & 15u;
                    if (!FLAGW) {
                        inner_bits = 0u;
#pragma unroll
                        for (int s = 0; s < NSUB; ++s) inner_bits |= ((ik[s] >> bit) & 1u) << s;
                    }
                    if (near)
                        sharp_fix<MODE, DT, GUARD, PHI, NSUB>(P, A, B, C, Xl, Yl, Zl, planar, inner_bits, cutb, tb, nm1,
                                                              nq, TX + oxi, TY + oyi, TZ + ozi, d);
#pragma unroll
                    for (int s = 0; s < NSUB; ++s) {
#pragma unroll
                        for (int t = 0; t < NX_LANE; ++t) {
                            const float dk = near ? d[4 * s + t] : 0.0f;
                            if (dk == 0.0f) continue;
                            const bool valid = (vmask >> (4 * s + t)) & 1u;
                            if (MODE == MODE_COUNT && valid) cnt += (dk > 0.0f) ? 1ull : ~0ull;
                            if (MODE == MODE_JT || MODE == MODE_COV) acc[s][t] = fmaf(dk, W, acc[s][t]);
                            if (MODE == MODE_J) part = fmaf(dk, mv[s][t], part);
                            if (MODE == MODE_JT4) {
#pragma unroll
                                for (int r = 0; r < 4; ++r) acc4[s & 1][t][r] = fmaf(dk, Wr[r], acc4[s & 1][t][r]);
                            }
                            if (MODE == MODE_J4) {
#pragma unroll
                                for (int r = 0; r < 4; ++r) part4[r] = fmaf(dk, mv4[s & 1][t][r], part4[r]);
                            }
                            if (MODE == MODE_FROB && valid) part += dk;
                        }
                    }
                }
                if (MODE == MODE_J) {
                    // Fold the row's 32 lane partials to 8 (lanes 0-7 then hold distinct sums)
                    // and park them in the row's own staged record, which every lane has read
                    // by now; the row's lane adds the 8 in a fixed order after the chunk.
                    part += __shfl_xor_sync(0xffffffffu, part, 16);
                    part += __shfl_xor_sync(0xffffffffu, part, 8);
                    __syncwarp();
                    if (lane < 8) reinterpret_cast<float*>(stg + bit * SR)[lane] = part;
                }
                if (MODE == MODE_J4) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float pr4 = warp_sum(part4[r]);
                        if (lane == bit) mypart4[r] = pr4 * W;
                    }
                }
                if (MODE == MODE_FROB) dacc += (double)part * (double)W * (double)W;
            }
            if (MODE == MODE_J) {
                __syncwarp();
                if (have) {
                    if (okb) {
                        const float4 r0 = stg[lane * SR + 0];
                        const float4 r1 = stg[lane * SR + 1];
                        const float Wl = stg[lane * SR + 2].x;
                        mypart = (r0.x + r0.y + r0.z + r0.w + r1.x + r1.y + r1.z + r1.w) * Wl;
                    }
                    P.vout[e * NREG + region] = mypart;
                }
            }
            if (MODE == MODE_J4 && have)
                *reinterpret_cast<float4*>(P.vout + (e * NREG + region) * 4) =
                    make_float4(mypart4[0], mypart4[1], mypart4[2], mypart4[3]);
            __syncwarp();
        }

        if (MODE == MODE_JT || MODE == MODE_COV) {
            const uint32_t vm = lane_vmask();
#pragma unroll
            for (int s = 0; s < NSUB; ++s) {
                const int dy = sub_dy<NSUB>(s), dz = sub_dz<NSUB>(s);
                if (item.slot < 0) {
#pragma unroll
                    for (int t = 0; t < NX_LANE; ++t)
                        if ((vm >> (4 * s + t)) & 1u)
                            P.vout[vbase + ((int64_t)dz * P.ny + dy) * P.nx + t] = acc[s][t];
                } else {
                    // local index inside the tile: (z * 16 + y) * 16 + x
                    const int loc = (((ozi + dz) * TILE_Y) + oyi + dy) * TILE_X + oxi;
                    float4 v4 = make_float4(acc[s][0], acc[s][1], acc[s][2], acc[s][3]);
                    *reinterpret_cast<float4*>(P.gpart + (int64_t)item.slot * TILE_VOX + loc) = v4;
                }
            }
        }
        if (MODE == MODE_JT4) {
            static_assert(!BATCH || NSUB == 2, "the four-column modes take 8 x 8 x 4 regions");
            const uint32_t vm = lane_vmask();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int loc = ((ozi * TILE_Y) + oyi + 4 * s) * TILE_X + oxi;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (item.slot < 0) {
#pragma unroll
                        for (int t = 0; t < NX_LANE; ++t)
                            if ((vm >> (4 * s + t)) & 1u)
                                P.vout[(int64_t)r * P.nvox + vbase + (int64_t)(4 * s) * P.nx + t] = acc4[s][t][r];
                    } else {
                        float4 v4 = make_float4(acc4[s][0][r], acc4[s][1][r], acc4[s][2][r], acc4[s][3][r]);
                        *reinterpret_cast<float4*>(P.gpart + ((int64_t)item.slot * 4 + r) * TILE_VOX + loc) = v4;
                    }
                }
            }
        }
        if (MODE == MODE_FROB) {
            dacc = warp_sum_d(dacc);
            if (lane == 0) P.dsum[unit] = dacc;
        }
        if (MODE == MODE_COUNT) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                cnt_eval += __shfl_xor_sync(0xffffffffu, cnt_eval, o);
            }
            if (lane == 0) {
                if (cnt) atomicAdd(P.icount, cnt);
                if (cnt_eval) atomicAdd(P.icount + 1, cnt_eval);
            }
        }
    }
}

// d_p = sum over the row's entries (ascending tile order) and the 4 regions of the partials.
__global__ void __launch_bounds__(256) j_reduce_kernel(const int64_t* __restrict__ row_off,
                                                       const int64_t* __restrict__ row_ent,
                                                       const float* __restrict__ jpart, int64_t M,
                                                       float* __restrict__ d) {
    // one warp per row: lane l takes the row's entries l, l + 32, ... in order (the 4 region
    // partials of an entry pairwise in FP32, entries accumulated in FP64), then a fixed
    // butterfly over the lanes; the order never depends on scheduling
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= M) return;
    double s = 0.0;
    const int64_t j1 = row_off[p + 1];
    int64_t j = row_off[p] + lane;
    for (; j + 32 < j1; j += 64) {   // two entries in flight, added in the same order
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(jpart + row_ent[j] * 4));
        const float4 a1 = __ldg(reinterpret_cast<const float4*>(jpart + row_ent[j + 32] * 4));
        s += (double)((a0.x + a0.y) + (a0.z + a0.w));
        s += (double)((a1.x + a1.y) + (a1.z + a1.w));
    }
    if (j < j1) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(jpart + row_ent[j] * 4));
        s += (double)((a.x + a.y) + (a.z + a.w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d[p] = (float)s;
}

// The four-column form of j_reduce_kernel: jpart4[(entry * 8 + region) * 4 + r]; the same lane
// order, pairing and butterfly per column, d[r * M + p].
__global__ void __launch_bounds__(256) j_reduce4_kernel(const int64_t* __restrict__ row_off,
                                                        const int64_t* __restrict__ row_ent,
                                                        const float* __restrict__ jpart4, int64_t M,
                                                        float* __restrict__ d) {
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= M) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t j1 = row_off[p + 1];
    for (int64_t j = row_off[p] + lane; j < j1; j += 32) {
        const float4* q = reinterpret_cast<const float4*>(jpart4 + row_ent[j] * 32);
        float4 g[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = __ldg(q + k);
        s[0] += (double)(((g[0].x + g[1].x) + (g[2].x + g[3].x)) + ((g[4].x + g[5].x) + (g[6].x + g[7].x)));
        s[1] += (double)(((g[0].y + g[1].y) + (g[2].y + g[3].y)) + ((g[4].y + g[5].y) + (g[6].y + g[7].y)));
        s[2] += (double)(((g[0].z + g[1].z) + (g[2].z + g[3].z)) + ((g[4].z + g[5].z) + (g[6].z + g[7].z)));
        s[3] += (double)(((g[0].w + g[1].w) + (g[2].w + g[3].w)) + ((g[4].w + g[5].w) + (g[6].w + g[7].w)));
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        double v = s[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) d[(int64_t)r * M + p] = (float)v;
    }
}

// g for voxels of tiles with several items (the slots summed in item order) or with none (0);
// tiles with one item were written by the apply kernel. One thread takes 4 consecutive x
// voxels of a tile (512 threads per tile); the slots are read 4 at a time so that several
// loads are in flight, and added one by one from 0 in slot order (deterministic).
// NCOL = 4: the four-column form, slot q of column r at gpart[((s0 + q) * 4 + r) * TILE_VOX],
// g[r * V + v].
template <int NCOL>
__global__ void __launch_bounds__(256) jt_reduce_kernel(const int32_t* __restrict__ slot0,
                                                        const int32_t* __restrict__ nslot,
                                                        const float* __restrict__ gpart, int64_t n_tiles, int nx,
                                                        int ny, int nz, int tiles_x, int tiles_y,
                                                        float* __restrict__ g) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_tiles * (TILE_VOX / 4)) return;
    const int T = (int)(idx / (TILE_VOX / 4));
    const int s0 = slot0[T];
    if (s0 == -1) return;
    const int loc = 4 * (int)(idx % (TILE_VOX / 4));
    const int ix = TILE_X * (T % tiles_x) + loc % TILE_X;
    const int iy = TILE_Y * ((T / tiles_x) % tiles_y) + (loc / TILE_X) % TILE_Y;
    const int iz = TILE_Z * (T / (tiles_x * tiles_y)) + loc / (TILE_X * TILE_Y);
    if (iy >= ny || iz >= nz || ix >= nx) return;
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t v = ((int64_t)iz * ny + iy) * nx + ix;
    const int ns = (s0 == -2) ? 0 : nslot[T];
#pragma unroll
    for (int r = 0; r < NCOL; ++r) {
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float* base = ns > 0 ? gpart + ((int64_t)s0 * NCOL + r) * TILE_VOX + loc : nullptr;
        int q = 0;
        for (; q + 4 <= ns; q += 4) {
            float4 w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)(q + k) * NCOL * TILE_VOX));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc.x += w[k].x;
                acc.y += w[k].y;
                acc.z += w[k].z;
                acc.w += w[k].w;
            }
        }
        for (; q < ns; ++q) {
            const float4 w = __ldcs(reinterpret_cast<const float4*>(base + (int64_t)q * NCOL * TILE_VOX));
            acc.x += w.x;
            acc.y += w.y;
            acc.z += w.z;
            acc.w += w.w;
        }
        float* out = g + (int64_t)r * V + v;
        out[0] = acc.x;
        if (ix + 1 < nx) out[1] = acc.y;
        if (ix + 2 < nx) out[2] = acc.z;
        if (ix + 3 < nx) out[3] = acc.w;
    }
}

static ApplyParams make_params(fft_geom g) {
    ApplyParams P;
    P.rec = g->rec;
    P.rec64 = g->rec64;
    P.row_band = g->row_band;
    P.tab = g->tab;
    P.n_bands = g->n_bands;
    P.n_tab = g->n_tab;
    P.bc = g->d_band;
    P.tile_rows = g->tile_rows;
    P.ebase = g->ebase;
    P.ebase3 = g->ebase3;
    P.items = g->items;
    P.n_items = g->n_items;
    P.counter = g->counter;
    P.tiles_x = g->tiles[0];
    P.tiles_y = g->tiles[1];
    P.nx = g->grid.nx;
    P.ny = g->grid.ny;
    P.nz = g->grid.nz;
    for (int a = 0; a < 3; ++a) P.org[a] = g->grid.origin[a];
    P.h = g->grid.h;
    P.vin = nullptr;
    P.vout = nullptr;
    P.gpart = g->gpart;
    P.dsum = nullptr;
    P.icount = nullptr;
    P.trig_nq = g->trig_nq;
    P.nvox = g->V;
    P.nrow = g->M;
    return P;
}

size_t apply_smem(fft_geom g, int warps) {
    size_t tab = ((size_t)g->n_bands * g->n_tab * sizeof(float2) + 15) & ~(size_t)15;
    return tab + (size_t)warps * STG_PER_WARP * sizeof(float4);
}

size_t apply_smem(fft_geom g) { return apply_smem(g, APPLY_WARPS); }

// Most warps (a multiple of 8, at most 24) one sharp-variant CTA can stage for.
static int sharp_max_warps(fft_geom g) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int w = SHARP_MAX_WARPS;
    while (w > APPLY_WARPS && apply_smem(g, w) > (size_t)optin) w -= 4;
    return w;
}

template <int MODE, int DT, bool G, bool S, int PHI>
static fft_status set_attr_one(size_t smem) {
    FFT_CUDA(cudaFuncSetAttribute(apply_kernel<MODE, DT, G, S, PHI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    return FFT_OK;
}

template <int MODE, int DT, int PHI>
static fft_status set_attr_dt(size_t smem) {
    fft_status rc;
    if ((rc = set_attr_one<MODE, DT, false, false, PHI>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_one<MODE, DT, true, false, PHI>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_one<MODE, DT, false, true, PHI>(smem)) != FFT_OK) return rc;
    return set_attr_one<MODE, DT, true, true, PHI>(smem);
}

template <int MODE>
static fft_status set_attr_mode(size_t smem) {
    fft_status rc;
    if ((rc = set_attr_dt<MODE, FFT_DT_STABLE, PHI_TABLE>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_dt<MODE, FFT_DT_NAIVE, PHI_TABLE>(smem)) != FFT_OK) return rc;
    if (MODE != MODE_COUNT && (rc = set_attr_dt<MODE, FFT_DT_STABLE, PHI_TRIG>(smem)) != FFT_OK) return rc;
    return set_attr_one<MODE, FFT_DT_FP64, false, false, PHI_TABLE>(smem);
}

// Most warps (at most 32) one plain wide CTA can stage for.
static int plain_max_warps(fft_geom g) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int w = PLAIN_MAX_WARPS;
    while (w > APPLY_WARPS && apply_smem(g, w) > (size_t)optin) w -= 8;
    return w;
}

// Raise the dynamic shared-memory limit of every kernel instantiation once per geometry
// (outside any stream capture), so launches need no attribute calls.
fft_status set_apply_attributes(fft_geom g) {
    const size_t smem = apply_smem(g, std::max(sharp_max_warps(g), plain_max_warps(g)));
    fft_status rc;
    if ((rc = set_attr_mode<MODE_JT>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_mode<MODE_J>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_mode<MODE_COUNT>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_mode<MODE_COV>(smem)) != FFT_OK) return rc;
    // batch modes: stable detour only (other geometries apply the columns one by one)
    if ((rc = set_attr_dt<MODE_JT4, FFT_DT_STABLE, PHI_TABLE>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_dt<MODE_JT4, FFT_DT_STABLE, PHI_TRIG>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_dt<MODE_J4, FFT_DT_STABLE, PHI_TABLE>(smem)) != FFT_OK) return rc;
    if ((rc = set_attr_dt<MODE_J4, FFT_DT_STABLE, PHI_TRIG>(smem)) != FFT_OK) return rc;
    return set_attr_mode<MODE_FROB>(smem);
}

// Persistent grid size: resident CTAs per SM of the J^T kernel times the SM count.
int apply_occupancy(fft_geom g) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_kernel<MODE_JT, FFT_DT_STABLE, false, false, PHI_TABLE>,
                                                  APPLY_THREADS, apply_smem(g));
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    return per_sm * sms;
}

// CTA shape of the sharp variants: the block of 8, 12, 16 or 20 warps with the most resident
// warps per SM (the smaller block on a tie), and the persistent grid that fills the GPU.
void sharp_launch_shape(fft_geom g) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    int best_w = APPLY_WARPS, best_b = 1, best_res = 0;
    for (int w = APPLY_WARPS; w <= sharp_max_warps(g); w += 4) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, apply_kernel<MODE_JT, FFT_DT_STABLE, false, true, PHI_TABLE>,
                                                      32 * w, apply_smem(g, w));
        if (b * w > best_res) {
            best_res = b * w;
            best_w = w;
            best_b = b;
        }
    }
    cudaGetLastError();
    g->sharp_warps = best_w;
    g->sharp_ctas = std::max(best_b, 1) * sms;
}

// CTA shape of the plain stable-detour table variants: 8-warp CTAs on the (autotuned)
// persistent grid, unless one wide CTA of 16, 24 or 32 warps keeps more warps resident per SM
// (large multi-band tables), then one such CTA per SM.
void plain_launch_shape(fft_geom g) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    int b8 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b8, apply_kernel<MODE_JT, FFT_DT_STABLE, false, false, PHI_TABLE>,
                                                  APPLY_THREADS, apply_smem(g));
    int best_w = APPLY_WARPS, best_b = std::max(b8, 1), best_res = b8 * APPLY_WARPS;
    for (int w = 2 * APPLY_WARPS; w <= plain_max_warps(g); w += APPLY_WARPS) {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, apply_kernel<MODE_JT, FFT_DT_STABLE, false, false, PHI_TABLE>,
                                                      32 * w, apply_smem(g, w));
        if (b * w > best_res) {
            best_res = b * w;
            best_w = w;
            best_b = b;
        }
    }
    cudaGetLastError();
    g->plain_warps = best_w;
    g->plain_ctas = std::max(best_b, 1) * sms;
}

// One apply launch over P's items: sharp single-column variants in the geometry's sharp CTA
// shape, plain stable-detour table variants in the plain shape, the others in 8-warp CTAs on
// the persistent grid.
template <int MODE, int DT, bool G, bool S, int PHI>
static void launch_apply(fft_geom g, const ApplyParams& P, cudaStream_t st) {
    if (apply_sharp_wide<MODE, DT, S, PHI>()) {
        apply_kernel<MODE, DT, G, S, PHI><<<g->sharp_ctas, 32 * g->sharp_warps, apply_smem(g, g->sharp_warps), st>>>(P);
    } else if (apply_plain_wide<MODE, DT, S, PHI>() && g->plain_warps > APPLY_WARPS) {
        apply_kernel<MODE, DT, G, S, PHI><<<g->plain_ctas, 32 * g->plain_warps, apply_smem(g, g->plain_warps), st>>>(P);
    } else {
        apply_kernel<MODE, DT, G, S, PHI><<<g->apply_ctas, APPLY_THREADS, apply_smem(g), st>>>(P);
    }
}

// A sharp geometry's plain items (rows of bands whose Phi vanishes at the cut) run in the plain
// variant, its sharp-band items in the sharp one: two launches, each pulling units from its own
// counter. Other geometries run all items in one launch.
template <int MODE, int DT, bool G, int PHI>
static void launch_split(fft_geom g, const ApplyParams& P, cudaStream_t st) {
    if (!g->sharp) {
        launch_apply<MODE, DT, G, false, PHI>(g, P, st);
        return;
    }
    const int np = g->n_items_plain, ns = g->n_items - g->n_items_plain;
    if (np > 0) {
        ApplyParams Q = P;
        Q.n_items = np;
        launch_apply<MODE, DT, G, false, PHI>(g, Q, st);
    }
    if (ns > 0) {
        ApplyParams Q = P;
        Q.items = P.items + np;
        Q.n_items = ns;
        Q.counter = P.counter + 1;
        if (Q.dsum) Q.dsum = P.dsum + (size_t)np * apply_regions<MODE>();   // per-unit partials follow the plain launch's
        launch_apply<MODE, DT, G, true, PHI>(g, Q, st);
    }
}

template <int MODE>
static fft_status launch_mode(fft_geom g, const ApplyParams& P, cudaStream_t st) {
    FFT_CUDA(cudaMemsetAsync(g->counter, 0, 2 * sizeof(int32_t), st));
    if (g->n_items == 0) return FFT_OK;
    // MODE_COUNT evaluates no Phi: the table variant serves both representations
    constexpr int PHI_T = MODE == MODE_COUNT ? PHI_TABLE : PHI_TRIG;
#define FFT_LAUNCH_GS(DTV, PV)                                      \
    do {                                                            \
        if (g->guard) launch_split<MODE, DTV, true, PV>(g, P, st);  \
        else launch_split<MODE, DTV, false, PV>(g, P, st);          \
    } while (0)
    if (g->phi_kind == PHI_TRIG) {   // geometry creation guarantees dt_mode STABLE
        FFT_LAUNCH_GS(FFT_DT_STABLE, PHI_T);
    } else if (g->dt_mode == FFT_DT_STABLE) {
        FFT_LAUNCH_GS(FFT_DT_STABLE, PHI_TABLE);
    } else if (g->dt_mode == FFT_DT_NAIVE) {
        FFT_LAUNCH_GS(FFT_DT_NAIVE, PHI_TABLE);
    } else {   // FP64 detour: the cut is decided in FP64 everywhere, one plain launch
        launch_apply<MODE, FFT_DT_FP64, false, false, PHI_TABLE>(g, P, st);
    }
#undef FFT_LAUNCH_GS
    FFT_CUDA(cudaGetLastError());
    return FFT_OK;
}

// The four-column modes (stable detour only).
template <int MODE>
static fft_status launch_batch(fft_geom g, const ApplyParams& P, cudaStream_t st) {
    const size_t smem = apply_smem(g);
    const int ctas = g->apply_ctas;
    FFT_CUDA(cudaMemsetAsync(g->counter, 0, sizeof(int32_t), st));
    if (g->n_items == 0) return FFT_OK;
#define FFT_LAUNCH(GV, SV, PV) apply_kernel<MODE, FFT_DT_STABLE, GV, SV, PV><<<ctas, APPLY_THREADS, smem, st>>>(P)
#define FFT_LAUNCH_GS(PV)                                           \
    do {                                                            \
        if (g->guard) {                                             \
            if (g->sharp) FFT_LAUNCH(true, true, PV);               \
            else FFT_LAUNCH(true, false, PV);                       \
        } else {                                                    \
            if (g->sharp) FFT_LAUNCH(false, true, PV);              \
            else FFT_LAUNCH(false, false, PV);                      \
        }                                                           \
    } while (0)
    if (g->phi_kind == PHI_TRIG)
        FFT_LAUNCH_GS(PHI_TRIG);
    else
        FFT_LAUNCH_GS(PHI_TABLE);
#undef FFT_LAUNCH_GS
#undef FFT_LAUNCH
    FFT_CUDA(cudaGetLastError());
    return FFT_OK;
}

static fft_status batch_scratch(fft_geom g) {
    if (!g->jpart4) {
        cudaError_t e = cudaMalloc(&g->jpart4, sizeof(float) * (size_t)(g->E > 0 ? g->E : 1) * 32);
        if (e == cudaSuccess && g->n_slots > 0)
            e = cudaMalloc(&g->gpart4, sizeof(float) * (size_t)g->n_slots * 4 * TILE_VOX);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(g->jpart4);
            g->jpart4 = nullptr;
            set_error("batch apply: cudaMalloc of the four-column scratch failed");
            return FFT_ERR_OOM;
        }
        g->scratch_bytes += (int64_t)(sizeof(float) * ((size_t)g->E * 32 + (size_t)g->n_slots * 4 * TILE_VOX));
    }
    return FFT_OK;
}

// d[:, c] = J m[:, c] for n columns: groups of four with the batch kernel on stable-detour
// geometries, single columns otherwise.
fft_status launch_J_batch(fft_geom g, const float* m, int n, float* d, cudaStream_t st) {
    int c = 0;
    if (g->dt_mode == FFT_DT_STABLE && n >= 4) {
        fft_status rc = batch_scratch(g);
        if (rc != FFT_OK) return rc;
        for (; c + 4 <= n; c += 4) {
            ApplyParams P = make_params(g);
            P.vin = m + (int64_t)c * g->V;
            P.vout = g->jpart4;
            if ((rc = launch_batch<MODE_J4>(g, P, st)) != FFT_OK) return rc;
            if (g->M > 0) {
                j_reduce4_kernel<<<(unsigned)ceil_div(g->M, 8), 256, 0, st>>>(g->row_off, g->row_ent, g->jpart4, g->M,
                                                                              d + (int64_t)c * g->M);
                FFT_CUDA(cudaGetLastError());
            }
        }
    }
    for (; c < n; ++c) {
        fft_status rc = launch_J(g, m + (int64_t)c * g->V, d + (int64_t)c * g->M, st);
        if (rc != FFT_OK) return rc;
    }
    return FFT_OK;
}

template <int NCOL>
static fft_status launch_jt_reduce(fft_geom g, const float* gpart, float* gout, cudaStream_t st) {
    const int64_t threads = g->n_tiles * (TILE_VOX / 4);
    if (threads == 0) return FFT_OK;
    jt_reduce_kernel<NCOL><<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(
        g->tile_slot0, g->tile_nslot, gpart, g->n_tiles, g->grid.nx, g->grid.ny, g->grid.nz, g->tiles[0],
        g->tiles[1], gout);
    FFT_CUDA(cudaGetLastError());
    return FFT_OK;
}

// g[:, c] = J^T d[:, c] for n columns (groups of four as above).
fft_status launch_JT_batch(fft_geom g, const float* din, int n, float* gout, cudaStream_t st) {
    int c = 0;
    if (g->dt_mode == FFT_DT_STABLE && n >= 4) {
        fft_status rc = batch_scratch(g);
        if (rc != FFT_OK) return rc;
        for (; c + 4 <= n; c += 4) {
            ApplyParams P = make_params(g);
            P.vin = din + (int64_t)c * g->M;
            P.vout = gout + (int64_t)c * g->V;
            P.gpart = g->gpart4;
            if ((rc = launch_batch<MODE_JT4>(g, P, st)) != FFT_OK) return rc;
            if ((rc = launch_jt_reduce<4>(g, g->gpart4, gout + (int64_t)c * g->V, st)) != FFT_OK) return rc;
        }
    }
    for (; c < n; ++c) {
        fft_status rc = launch_JT(g, din + (int64_t)c * g->M, gout + (int64_t)c * g->V, st);
        if (rc != FFT_OK) return rc;
    }
    return FFT_OK;
}

fft_status launch_J(fft_geom g, const float* m, float* d, cudaStream_t st) {
    ApplyParams P = make_params(g);
    P.vin = m;
    P.vout = g->jpart;
    fft_status rc = launch_mode<MODE_J>(g, P, st);
    if (rc != FFT_OK) return rc;
    if (g->M > 0) {
        int64_t blocks = ceil_div(g->M, 8);   // 8 rows (warps) per block
        j_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(g->row_off, g->row_ent, g->jpart, g->M, d);
        FFT_CUDA(cudaGetLastError());
    }
    return FFT_OK;
}

fft_status launch_JT(fft_geom g, const float* din, float* gout, cudaStream_t st) {
    ApplyParams P = make_params(g);
    P.vin = din;
    P.vout = gout;
    fft_status rc = launch_mode<MODE_JT>(g, P, st);
    if (rc != FFT_OK) return rc;
    return launch_jt_reduce<1>(g, g->gpart, gout, st);
}

// cov_v = sum_p |J[p, v] w_p| (w null: all ones), gathered like J^T.
fft_status launch_cov(fft_geom g, const float* w, float* cov, cudaStream_t st) {
    ApplyParams P = make_params(g);
    P.vin = w;
    P.vout = cov;
    fft_status rc = launch_mode<MODE_COV>(g, P, st);
    if (rc != FFT_OK) return rc;
    return launch_jt_reduce<1>(g, g->gpart, cov, st);
}

// In-support evaluations (dt < dt_max) of one apply and evaluations actually performed.
fft_status count_support(fft_geom g, int64_t* support, int64_t* evaluated) {
    ApplyParams P = make_params(g);
    unsigned long long* d_cnt = nullptr;
    FFT_CUDA(cudaMalloc(&d_cnt, 2 * sizeof(unsigned long long)));
    cudaError_t e0 = cudaMemset(d_cnt, 0, 2 * sizeof(unsigned long long));
    if (e0 != cudaSuccess) {
        cudaFree(d_cnt);
        return cuda_fail(e0, "count_support: cudaMemset");
    }
    P.icount = d_cnt;
    fft_status rc = launch_mode<MODE_COUNT>(g, P, 0);
    unsigned long long h[2] = {0, 0};
    if (rc == FFT_OK) {
        cudaError_t e = cudaMemcpy(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "count_support");
    }
    cudaFree(d_cnt);
    *support = (int64_t)h[0];
    *evaluated = (int64_t)h[1];
    return rc;
}

fft_status compute_frob2(fft_geom g, double* out) {
    ApplyParams P = make_params(g);
    double* d_sum = nullptr;
    size_t n = (size_t)(g->n_items > 0 ? g->n_items : 1) * APPLY_WARPS;   // one per unit
    FFT_CUDA(cudaMalloc(&d_sum, n * sizeof(double)));
    cudaError_t e0 = cudaMemset(d_sum, 0, n * sizeof(double));
    if (e0 != cudaSuccess) {
        cudaFree(d_sum);
        return cuda_fail(e0, "frob2: cudaMemset");
    }
    P.dsum = d_sum;
    fft_status rc = launch_mode<MODE_FROB>(g, P, 0);
    std::vector<double> h(n, 0.0);
    if (rc == FFT_OK) {
        cudaError_t e = cudaMemcpy(h.data(), d_sum, n * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "frob2");
    }
    cudaFree(d_sum);
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += h[i];
    *out = s;
    return rc;
}

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_J_apply(fft_geom g, const float* m_dev, float* d_dev, void* stream) {
    FFT_API_RANGE("fft_J_apply");
    FFT_ARG(g && m_dev && d_dev, "fft_J_apply: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    return launch_J(g, m_dev, d_dev, (cudaStream_t)stream);
}

extern "C" fft_status fft_JT_apply(fft_geom g, const float* d_dev, float* g_dev, void* stream) {
    FFT_API_RANGE("fft_JT_apply");
    FFT_ARG(g && d_dev && g_dev, "fft_JT_apply: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    return launch_JT(g, d_dev, g_dev, (cudaStream_t)stream);
}

extern "C" fft_status fft_J_apply_batch(fft_geom g, const float* m_dev, int32_t n, float* d_dev, void* stream) {
    FFT_API_RANGE("fft_J_apply_batch");
    FFT_ARG(g && m_dev && d_dev, "fft_J_apply_batch: null argument");
    FFT_ARG(n >= 1, "fft_J_apply_batch: need n >= 1 columns");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    return launch_J_batch(g, m_dev, n, d_dev, (cudaStream_t)stream);
}

extern "C" fft_status fft_JT_apply_batch(fft_geom g, const float* d_dev, int32_t n, float* g_dev, void* stream) {
    FFT_API_RANGE("fft_JT_apply_batch");
    FFT_ARG(g && d_dev && g_dev, "fft_JT_apply_batch: null argument");
    FFT_ARG(n >= 1, "fft_JT_apply_batch: need n >= 1 columns");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    return launch_JT_batch(g, d_dev, n, g_dev, (cudaStream_t)stream);
}

extern "C" fft_status fft_coverage(fft_geom g, const float* w_dev, float* cov_dev, void* stream) {
    FFT_API_RANGE("fft_coverage");
    FFT_ARG(g && cov_dev, "fft_coverage: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    return launch_cov(g, w_dev, cov_dev, (cudaStream_t)stream);
}

extern "C" fft_status fft_frob2(fft_geom g, double* out) {
    FFT_API_RANGE("fft_frob2");
    FFT_ARG(g && out, "fft_frob2: null argument");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    if (g->frob2 < 0.0) {
        double v = 0.0;
        rc = compute_frob2(g, &v);
        if (rc != FFT_OK) return rc;
        g->frob2 = v;
    }
    *out = g->frob2;
    return FFT_OK;
}
