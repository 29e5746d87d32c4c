// Batched Hessian point-spread functions on the tensor cores (Sec. II-D, Eq. resolution_2):
//
//   Y[v, j] = sum_p J[p, v] D[p, j],   D[p, j] = J[p, spike_k] [p in S_s],  j = s * n_spike + k
//
// i.e. Y = J^T D with many right-hand sides, which is a dense contraction per voxel block:
// for an 8 x 4 x 4 sub-brick (128 voxels = the MMA's M) the rows whose support reaches it are
// the contraction dimension K and the (subset, spike) columns are N.
//
// Per CTA (one per SM; 16 generator warps and one MMA warp) and sub-brick:
//   1. scan the tile's candidate rows, keep those that may reach the sub-brick (tangent-plane
//      bound of the convex detour), stage their pair-frame data in shared memory;
//   2. for every chunk of 32 kept rows, generator warp w owns rows 2w and 2w + 1: it clears the
//      sparse D entries it wrote into the chunk's B buffer three chunks earlier, scatters the
//      rows' D entries (BF16), generates its two rows of the A tile J[p, v] (FP32 evaluation as
//      in the J^T kernel, rounded to BF16) and arrives on the buffer's "full" mbarrier; the MMA
//      warp waits for it, issues tcgen05.mma (M = 128, N = up to 2 x 256, K = 32) accumulating
//      in TMEM and commits to the buffer's "empty" mbarrier, which the generators wait for
//      before they reuse the buffer. Three A / B buffers and no CTA-wide barrier per chunk let
//      generation run up to three chunks ahead of the tensor cores;
//   3. after the last chunk, TMEM -> registers -> Y.
// Every wait is bounded; a thread whose wait timed out sets a status word and waits no more,
// and the CTA stops at the end of the sub-brick.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fft_common.cuh"
#include "fft_device.cuh"
#include "fft_tc.cuh"

namespace fftgb {

namespace {

constexpr int GEN_WARPS = 16;          // warps that generate J and scatter D
constexpr int TC_WARPS = GEN_WARPS + 1;    // + one warp that issues the MMAs
constexpr int TC_THREADS = TC_WARPS * 32;
constexpr int KC = 32;                 // rows per chunk (MMA K per chunk): 2 per generator warp
constexpr int NSTAGE = 3;              // A / B buffers in the ring
constexpr int SEG = TC_THREADS;        // tile entries scanned per pass (one per thread)
constexpr int LIST_CAP = SEG + KC;     // kept rows waiting for a chunk (staged records)
constexpr int D_LANES = 16;            // lanes that scatter one row's D entries
constexpr long long WAIT_BUDGET = 4000000000ll;   // cycles (~2 s)

struct PsfTcParams {
    const RowRec* rec;
    const int32_t* row_band;
    const BandConst* bc;
    const float2* tab;
    int n_bands, n_tab;
    const int32_t* tile_rows;
    const int64_t* tile_off;
    const float4* ebase;
    const float* ebase3;
    const int32_t* units;      // (tile << 4) | sub-brick, heaviest tiles first
    int n_units;
    int32_t* counter;
    int tiles_x, tiles_y;
    int nx, ny, nz;
    const int64_t* d_off;      // sparse D rows: [M + 1]
    const uint16_t* d_idx;     // column j
    const float* d_val;
    int n_rhs;                 // columns of D / Y
    const int32_t* col_map;    // output column of each D column
    int n_half;                // N of one MMA (multiple of 16, <= 256)
    int nh;                    // MMAs per K step (1 or 2)
    int b_rows;                // rows of the B tile (nh * n_half)
    int tmem_cols;
    float* out;                // Y as out[j * V + v]
    int64_t V;
    int32_t* status;
    unsigned long long* chunks;   // chunks (128 x 32 A tiles) issued, summed over CTAs
};

struct TcShared {
    unsigned long long full[NSTAGE];    // generator warps -> MMA warp (GEN_WARPS arrivals)
    unsigned long long empty[NSTAGE];   // MMA warp -> generator warps (tcgen05.commit)
    uint32_t tmem_slot;
    int unit;
    int wcnt[TC_WARPS];
};

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(mbar, parity)) {
        if (clock64() - t0 > WAIT_BUDGET) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// GUARD: some voxel centre lies on a transducer (the geometry's flag): the guarded detour.
template <bool GUARD>
__global__ void __launch_bounds__(TC_THREADS, 1) psf_tc_kernel(const __grid_constant__ PsfTcParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcShared S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool is_gen = warp < GEN_WARPS;

    // ---- shared-memory carve-up: A[NSTAGE], B[NSTAGE] (1 KB aligned), table, staged row list
    const uint32_t a_bytes = 128u * KC * 2u;
    const uint32_t b_bytes = (uint32_t)P.b_rows * KC * 2u;
    unsigned char* sA0 = smem;
    unsigned char* sB0 = smem + NSTAGE * a_bytes;
    size_t off = NSTAGE * (size_t)a_bytes + NSTAGE * (size_t)b_bytes;
    float2* s_tab = reinterpret_cast<float2*>(smem + off);
    off += ((size_t)P.n_bands * P.n_tab * sizeof(float2) + 15) & ~(size_t)15;
    float4* s_stg = reinterpret_cast<float4*>(smem + off);          // [LIST_CAP][3] staged kept rows

    for (int i = tid; i < P.n_bands * P.n_tab; i += TC_THREADS) s_tab[i] = P.tab[i];
    {   // B buffers start cleared; afterwards each generator lane clears the entries it wrote
        uint4* b4 = reinterpret_cast<uint4*>(sB0);
        for (uint32_t i = tid; i < NSTAGE * b_bytes / 16; i += TC_THREADS) b4[i] = make_uint4(0, 0, 0, 0);
    }
    const uint32_t tab_addr = smem_addr(s_tab);
    const float nm1 = (float)(P.n_tab - 1);
    const uint32_t full0 = smem_addr(&S.full[0]), empty0 = smem_addr(&S.empty[0]);
    if (warp == 0) {
        tc::tmem_alloc(smem_addr(&S.tmem_slot), (uint32_t)P.tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < NSTAGE; ++b) {
            tc::mbar_init(full0 + 8u * b, GEN_WARPS);
            tc::mbar_init(empty0 + 8u * b, 1);
        }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = S.tmem_slot;
    const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)P.n_half);

    int chunk = 0;        // chunks issued by this CTA so far (selects buffer and mbarrier phases)
    bool failed = false;
    // Generation role: warp w evaluates rows 2w and 2w + 1 of a chunk; lane l owns the four
    // consecutive x voxels (4 lx + t, ly, lz), t = 0..3, of the 8 x 4 x 4 sub-brick, with
    // lx = l & 1, ly = (l >> 1) & 3, lz = l >> 3. Voxel t of lane l is MMA row (TMEM lane)
    // m = 32 t + l, which spreads a warp's stores over all eight 16-byte slots of a core matrix.
    // For D the warp owns B-tile rows 2w (lanes 0-15) and 2w + 1 (lanes 16-31) of every buffer;
    // lane i of a half scatters the row's D entries i and i + 16 (more, rarely, in a loop).
    const int glx = lane & 1, gly = (lane >> 1) & 3, glz = lane >> 3;
    const int d_r = 2 * warp + (lane >> 4), d_i0 = lane & (D_LANES - 1);
    // D positions this lane wrote into the buffer of the current chunk, of the next one and of
    // the one after (the buffers rotate with the chunks): (j0 + 1) | (j1 + 1) << 10, bit 20 if
    // the row had more than 2 D_LANES entries (then the lane clears its whole share of the row)
    uint32_t old0 = 0, old1 = 0, old2 = 0;

    for (;;) {
        __syncthreads();   // everyone has read the previous unit index before it is replaced
        if (tid == 0) S.unit = atomicAdd(P.counter, 1);
        __syncthreads();
        const int unit = S.unit;
        if (unit >= P.n_units || failed) break;
        const int T = P.units[unit] >> 4, sb = P.units[unit] & 15;
        const int tx = T % P.tiles_x, ty = (T / P.tiles_x) % P.tiles_y, tz = T / (P.tiles_x * P.tiles_y);
        // sub-brick origin in the tile (8 x 4 x 4 bricks: 2 along x, 4 along y, 2 along z)
        const int SX = 8 * (sb & 1), SY = 4 * ((sb >> 1) & 3), SZ = 4 * (sb >> 3);
        const int X0 = TILE_X * tx + SX, Y0 = TILE_Y * ty + SY, Z0 = TILE_Z * tz + SZ;
        if (X0 >= P.nx || Y0 >= P.ny || Z0 >= P.nz) continue;   // uniform across the CTA
        const int64_t e_begin = P.tile_off[T], e_end = P.tile_off[T + 1];
        // this lane's first voxel, relative to the tile origin (generation)
        const float Xv = (float)(SX + 4 * glx), Yv = (float)(SY + gly), Zv = (float)(SZ + glz);
        int n_list = 0, head = 0, unit_chunks = 0;

        for (int64_t seg = e_begin; seg < e_end; seg += SEG) {
            // ---- 1. scan: keep rows that may reach the sub-brick, staged in the row list;
            //         the rows left over from the previous pass move to the front first
            __syncthreads();   // every warp is done with the list entries of earlier chunks
            if (head > 0) {
                const int carry = n_list - head;
                float4 c0, c1, c2;
                if (tid < carry) {
                    c0 = s_stg[(head + tid) * 3 + 0];
                    c1 = s_stg[(head + tid) * 3 + 1];
                    c2 = s_stg[(head + tid) * 3 + 2];
                }
                __syncthreads();
                if (tid < carry) {
                    s_stg[tid * 3 + 0] = c0;
                    s_stg[tid * 3 + 1] = c1;
                    s_stg[tid * 3 + 2] = c2;
                }
                n_list = carry;
                head = 0;
            }
            {
                const int64_t e = seg + tid;
                bool keep = false;
                float4 s0, s1, s2;
                if (e < e_end) {
                    const int p = P.tile_rows[e];
                    const int64_t d0 = P.d_off[p], d1 = P.d_off[p + 1];
                    if (d1 > d0) {   // rows without D entries add nothing
                        const RowRec r = P.rec[p];
                        const int b = P.row_band[p];
                        const BandConst bc = P.bc[b];
                        const float hb = bc.h;
                        const float ex = r.b.x, ey = r.b.y, ez = r.b.z, hl = r.a.w;
                        const float cx = fmaf((float)(X0) + 3.5f, hb, bc.org[0]) - r.a.x;
                        const float cy = fmaf((float)(Y0) + 1.5f, hb, bc.org[1]) - r.a.y;
                        const float cz = fmaf((float)(Z0) + 1.5f, hb, bc.org[2]) - r.a.z;
                        keep = box_may_touch(cx, cy, cz, ex, ey, ez, hl, 3.5f * hb, 1.5f * hb, 1.5f * hb);
                        if (keep) {
                            // is the whole sub-brick between the transducer planes? a planar pair?
                            const float pext = 3.5f * hb * fabsf(ex) + 1.5f * hb * (fabsf(ey) + fabsf(ez)) + 1e-3f;
                            const bool inner = fabsf(fmaf(cx, ex, fmaf(cy, ey, cz * ez))) + pext <= hl;
                            // table base (a multiple of 8) with the inner / planar flags in bits 0, 1
                            const uint32_t tb = (tab_addr + (uint32_t)(b * P.n_tab) * 8u - MAGIC_BITS_X8) |
                                                (inner ? 1u : 0u) | (ez == 0.0f ? 2u : 0u);
                            s0 = P.ebase[e];
                            s1 = make_float4(hb * ex, hb * ey, hb * ez, P.ebase3[e]);
                            s2 = make_float4(r.b.w, __uint_as_float(tb), __uint_as_float((uint32_t)d0),
                                             __int_as_float((int)(d1 - d0)));
                        }
                    }
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) S.wcnt[warp] = __popc(bal);
                __syncthreads();
                int before = 0, total = 0;
#pragma unroll
                for (int w = 0; w < TC_WARPS; ++w) {
                    const int c = S.wcnt[w];
                    before += (w < warp) ? c : 0;
                    total += c;
                }
                if (keep) {
                    const int pos = n_list + before + __popc(bal & ((1u << lane) - 1u));
                    s_stg[pos * 3 + 0] = s0;
                    s_stg[pos * 3 + 1] = s1;
                    s_stg[pos * 3 + 2] = s2;
                }
                n_list += total;
                __syncthreads();
            }
            const bool last_seg = seg + SEG >= e_end;
            // ---- 2. chunks of KC kept rows: no CTA-wide barrier, only the two mbarrier rings
            while (n_list - head >= KC || (last_seg && n_list - head > 0)) {
                const int nrows = min(KC, n_list - head);
                const int buf = chunk % NSTAGE;
                const uint32_t use = (uint32_t)(chunk / NSTAGE);   // use count of this buffer
                unsigned char* sA = sA0 + buf * a_bytes;
                unsigned char* sB = sB0 + buf * b_bytes;
                if (is_gen) {
                    const float4* stg = s_stg + (size_t)head * 3;
                    if (chunk >= NSTAGE && !failed) {   // the MMAs that last read this buffer must be done
                        if (!wait_phase(empty0 + 8u * buf, (use - 1u) & 1u)) {
                            if (lane == 0) atomicExch(P.status, FFT_ERR_TIMEOUT);
                            failed = true;
                        }
                    }
                    // D entries of this lane's B row: loads issued now, stored after the generation
                    uint32_t d_beg = 0;
                    int d_cnt = 0;
                    if (d_r < nrows) {
                        const float4 C = stg[d_r * 3 + 2];
                        d_beg = __float_as_uint(C.z);
                        d_cnt = __float_as_int(C.w);
                    }
                    const bool has0 = d_i0 < d_cnt, has1 = d_i0 + D_LANES < d_cnt;
                    uint32_t j0 = 0, j1 = 0;
                    float dv0 = 0.0f, dv1 = 0.0f;
                    if (has0) {
                        j0 = P.d_idx[d_beg + d_i0];
                        dv0 = P.d_val[d_beg + d_i0];
                    }
                    if (has1) {
                        j1 = P.d_idx[d_beg + d_i0 + D_LANES];
                        dv1 = P.d_val[d_beg + d_i0 + D_LANES];
                    }
                    // generate A: rows 2 warp, 2 warp + 1; this lane's four voxels
                    float vals[2][NX_LANE];
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr) {
                        const int r = 2 * warp + rr;
                        if (r < nrows) {
                            const float4 A4 = stg[r * 3 + 0];
                            const float4 B4 = stg[r * 3 + 1];
                            const float4 C4 = stg[r * 3 + 2];
                            const float hx = B4.x, hy = B4.y, hz = B4.z;
                            const float o = fmaf(Xv, hx, fmaf(Yv, hy, Zv * hz));
                            const float psb = A4.x + o, prb = A4.y + o;
                            const float c1 = fmaf(Yv, hz, fmaf(-Zv, hy, A4.z));
                            const float c2 = fmaf(Zv, hx, fmaf(-Xv, hz, A4.w));
                            const float c3 = fmaf(Xv, hy, fmaf(-Yv, hx, B4.w));
                            const float c1sq = c1 * c1;
                            const float c12sq = fmaf(c2, c2, c1sq);
                            const uint32_t tbf = __float_as_uint(C4.y);
                            const uint32_t tb = tbf & ~3u;
                            // warp-uniform choice of the detour form for the whole run of voxels
#define FFT_TC_RUN(INNER_V, PLANAR_V)                                                              \
    _Pragma("unroll") for (int t = 0; t < NX_LANE; ++t) {                                        \
        const float ft = (float)t;                                                               \
        const float pst = (t == 0 ? psb : fmaf(ft, hx, psb)), prt = (t == 0 ? prb : fmaf(ft, hx, prb)); \
        const float c3t = (t == 0 ? c3 : fmaf(ft, hy, c3));                                        \
        float q2;                                                                                \
        if (PLANAR_V) {                                                                          \
            q2 = fmaf(c3t, c3t, c12sq);                                                          \
        } else {                                                                                 \
            const float c2t = (t == 0 ? c2 : fmaf(-ft, hz, c2));                                   \
            q2 = fmaf(c2t, c2t, fmaf(c3t, c3t, c1sq));                                           \
        }                                                                                        \
        float is, ir;                                                                            \
        const float v = detour_v<FFT_DT_STABLE, GUARD, INNER_V>(pst, prt, q2, 0.0f, is, ir);     \
        vals[rr][t] = phi_lookup(v, tb, nm1) * (is * ir) * C4.x;                                 \
    }
                            if (tbf & 1u) {
                                if (tbf & 2u) {
                                    FFT_TC_RUN(true, true)
                                } else {
                                    FFT_TC_RUN(true, false)
                                }
                            } else {
                                if (tbf & 2u) {
                                    FFT_TC_RUN(false, true)
                                } else {
                                    FFT_TC_RUN(false, false)
                                }
                            }
#undef FFT_TC_RUN
                        } else {
#pragma unroll
                            for (int t = 0; t < NX_LANE; ++t) vals[rr][t] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int t = 0; t < NX_LANE; ++t)
                        *reinterpret_cast<uint32_t*>(sA + tc::kmajor_offset((uint32_t)(32 * t + lane),
                                                                            (uint32_t)(2 * warp), KC)) =
                            pack_bf16x2(vals[0][t], vals[1][t]);
                    // B: clear what this lane wrote into the buffer three chunks ago, then scatter
                    if (old0 & (1u << 20)) {
                        for (int j = d_i0; j < P.b_rows; j += D_LANES)
                            *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset((uint32_t)j, (uint32_t)d_r, KC)) = 0;
                    } else {
                        if (old0 & 0x3FFu)
                            *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset((old0 & 0x3FFu) - 1u, (uint32_t)d_r, KC)) = 0;
                        if ((old0 >> 10) & 0x3FFu)
                            *reinterpret_cast<uint16_t*>(
                                sB + tc::kmajor_offset(((old0 >> 10) & 0x3FFu) - 1u, (uint32_t)d_r, KC)) = 0;
                    }
                    __syncwarp();   // another lane of the half may write where this one cleared
                    if (has0)
                        *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(j0, (uint32_t)d_r, KC)) =
                            __float2bfloat16_rn(dv0);
                    if (has1)
                        *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset(j1, (uint32_t)d_r, KC)) =
                            __float2bfloat16_rn(dv1);
                    for (int i = d_i0 + 2 * D_LANES; i < d_cnt; i += D_LANES)   // long rows (rare)
                        *reinterpret_cast<__nv_bfloat16*>(sB + tc::kmajor_offset((uint32_t)P.d_idx[d_beg + i],
                                                                                 (uint32_t)d_r, KC)) =
                            __float2bfloat16_rn(P.d_val[d_beg + i]);
                    const uint32_t now = d_cnt > 2 * D_LANES ? (1u << 20)
                                                             : (has0 ? j0 + 1u : 0u) | ((has1 ? j1 + 1u : 0u) << 10);
                    old0 = old1;
                    old1 = old2;
                    old2 = now;
                    // publish this warp's part of the chunk to the MMA warp
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(full0 + 8u * buf);
                } else if (lane == 0) {
                    // MMA warp: wait until all generator warps have written the chunk, then issue
                    if (!failed && !wait_phase(full0 + 8u * buf, use & 1u)) {
                        atomicExch(P.status, FFT_ERR_TIMEOUT);
                        failed = true;
                    }
                    tc::fence_after_sync();
                    const uint32_t a_base = smem_addr(sA), b_base = smem_addr(sB);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint64_t ad = tc::smem_desc(a_base + 256u * ks, 128u, 16u * KC);
                        for (int h = 0; h < P.nh; ++h) {
                            const uint64_t bd =
                                tc::smem_desc(b_base + (uint32_t)(h * P.n_half) * (KC * 2u) + 256u * ks, 128u, 16u * KC);
                            tc::mma_bf16(taddr + (uint32_t)(h * P.n_half), ad, bd, idesc,
                                         (unit_chunks > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(empty0 + 8u * buf);
                }
                ++chunk;
                ++unit_chunks;
                head += nrows;
            }
        }
        if (__syncthreads_or(failed)) break;
        if (unit_chunks == 0) continue;
        // ---- 3. all MMAs of this unit done -> TMEM -> Y
        {
            const int last = chunk - 1;
            if (!wait_phase(empty0 + 8u * (last % NSTAGE), (uint32_t)((last / NSTAGE) & 1))) {
                if (tid == 0) atomicExch(P.status, FFT_ERR_TIMEOUT);
                failed = true;
            }
        }
        if (__syncthreads_or(failed)) break;
        tc::fence_after_sync();
        if (is_gen) {
            const int quarter = warp & 3;              // TMEM lanes this warp may access
            // TMEM lane 32 quarter + lane holds voxel t = quarter of generation lane `lane`
            const int x = X0 + 4 * (lane & 1) + quarter, y = Y0 + ((lane >> 1) & 3), z = Z0 + (lane >> 3);
            const bool valid = x < P.nx && y < P.ny && z < P.nz;
            const int64_t v = ((int64_t)z * P.ny + y) * P.nx + x;
            const int cols = P.nh * P.n_half;
            for (int c = 8 * (warp >> 2); c < cols; c += 32) {
                float vals[8];
                tc::tmem_ld_x8(taddr + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c, vals);
                if (valid) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (c + i < P.n_rhs) P.out[(int64_t)P.col_map[c + i] * P.V + v] = vals[i];
                }
            }
        }
        tc::fence_before_sync();
    }
    // drain: every issued MMA must be complete before the accumulator is released
    if (chunk > 0) {   // MMAs complete in order: the last one done means all are done
        const int last = chunk - 1;
        wait_phase(empty0 + 8u * (last % NSTAGE), (uint32_t)((last / NSTAGE) & 1));
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tmem_cols);
    if (tid == 0 && chunk > 0) atomicAdd(P.chunks, (unsigned long long)chunk);
}

}  // namespace

static size_t psf_tc_smem(fft_geom g, int b_rows) {
    return NSTAGE * (size_t)(128 * KC * 2) + NSTAGE * (size_t)b_rows * KC * 2 +
           (((size_t)g->n_bands * g->n_tab * sizeof(float2) + 15) & ~(size_t)15) +
           (size_t)LIST_CAP * 3 * sizeof(float4) + sizeof(TcShared) + 1024;
}

// Largest number of right-hand sides one tensor-core launch can take on this device (the B
// ring grows with it): a multiple of 16, at most 512; 0 if even 16 do not fit.
int psf_tc_max_cols(fft_geom g) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 0;
    for (int c = 16; c <= 512; c += 16) {
        const int nh = c > 256 ? 2 : 1;
        const int n_half = (int)ceil_div(ceil_div(c, nh), 16) * 16;
        if (psf_tc_smem(g, nh * n_half) <= (size_t)optin) best = c;
    }
    return best;
}

// Y = J^T D on the tensor cores for D given as sparse rows (d_off, d_idx, d_val) with n_rhs
// columns (1 .. 512); column j of Y goes to out[col_map[j] * V + v]. out must be zeroed by the
// caller (voxels that no row reaches are not written). Synchronous; returns FFT_ERR_TIMEOUT if
// a bounded wait gave up.
fft_status launch_psf_tc(fft_geom g, const int64_t* d_off, const uint16_t* d_idx, const float* d_val, int n_rhs,
                         const int32_t* col_map, float* out, cudaStream_t st) {
    if (n_rhs < 1 || n_rhs > 512) {
        set_error("psf tensor-core path: 1 .. 512 right-hand sides per launch");
        return FFT_ERR_ARG;
    }
    if (g->E == 0) return FFT_OK;
    const int nh = n_rhs > 256 ? 2 : 1;
    const int n_half = (int)ceil_div(ceil_div(n_rhs, nh), 16) * 16;
    int cols = nh * n_half, tmem_cols = 32;
    while (tmem_cols < cols) tmem_cols <<= 1;

    // units: the 16 sub-bricks of every tile with candidate rows, heaviest tiles first
    std::vector<int64_t> toff(g->n_tiles + 1);
    FFT_CUDA(cudaMemcpy(toff.data(), g->tile_off, sizeof(int64_t) * (g->n_tiles + 1), cudaMemcpyDeviceToHost));
    std::vector<int32_t> tiles;
    for (int64_t T = 0; T < g->n_tiles; ++T)
        if (toff[T + 1] > toff[T]) tiles.push_back((int32_t)T);
    std::stable_sort(tiles.begin(), tiles.end(),
                     [&](int32_t a, int32_t b) { return toff[a + 1] - toff[a] > toff[b + 1] - toff[b]; });
    std::vector<int32_t> units;
    units.reserve(tiles.size() * 16);
    for (int32_t T : tiles)
        for (int s = 0; s < 16; ++s) units.push_back((T << 4) | s);
    if (units.empty()) return FFT_OK;

    int32_t *d_units = nullptr, *d_ctr = nullptr;
    FFT_CUDA(cudaMalloc(&d_units, sizeof(int32_t) * units.size()));
    cudaError_t e = cudaMalloc(&d_ctr, 4 * sizeof(int32_t));   // counter, status, 64-bit chunk count
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_units, units.data(), sizeof(int32_t) * units.size(),
                                              cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, 4 * sizeof(int32_t), st);

    PsfTcParams P;
    P.rec = g->rec;
    P.row_band = g->row_band;
    P.bc = g->d_band;
    P.tab = g->tab;
    P.n_bands = g->n_bands;
    P.n_tab = g->n_tab;
    P.tile_rows = g->tile_rows;
    P.tile_off = g->tile_off;
    P.ebase = g->ebase;
    P.ebase3 = g->ebase3;
    P.units = d_units;
    P.n_units = (int)units.size();
    P.counter = d_ctr;
    P.tiles_x = g->tiles[0];
    P.tiles_y = g->tiles[1];
    P.nx = g->grid.nx;
    P.ny = g->grid.ny;
    P.nz = g->grid.nz;
    P.d_off = d_off;
    P.d_idx = d_idx;
    P.d_val = d_val;
    P.n_rhs = n_rhs;
    P.col_map = col_map;
    P.n_half = n_half;
    P.nh = nh;
    P.b_rows = nh * n_half;
    P.tmem_cols = tmem_cols;
    P.out = out;
    P.V = g->V;
    P.status = d_ctr + 1;
    P.chunks = reinterpret_cast<unsigned long long*>(d_ctr + 2);

    // at least 120 KB so that only one CTA (which holds TMEM for the whole launch) fits on an SM
    const size_t smem = std::max<size_t>(120 * 1024, psf_tc_smem(g, P.b_rows) - sizeof(TcShared) - 1024);
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && smem + sizeof(TcShared) > (size_t)optin) {
        cudaFree(d_units);
        cudaFree(d_ctr);
        set_error("psf tensor-core path: tables and tiles do not fit in shared memory");
        return FFT_ERR_ARG;
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(g->guard ? psf_tc_kernel<true> : psf_tc_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        if (g->guard)
            psf_tc_kernel<true><<<sms, TC_THREADS, smem, st>>>(P);
        else
            psf_tc_kernel<false><<<sms, TC_THREADS, smem, st>>>(P);
        e = cudaGetLastError();
    }
    int32_t hs[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, d_ctr, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int32_t status = hs[1];
    unsigned long long nch = 0;
    memcpy(&nch, hs + 2, sizeof(nch));
    // MMA work of this launch: every chunk multiplies a 128 x 32 BF16 tile by 32 x cols
    g->psf_tc_mma_flops += 2.0 * 128.0 * KC * (double)cols * (double)nch;
    cudaFree(d_units);
    cudaFree(d_ctr);
    if (e != cudaSuccess) return cuda_fail(e, "psf tensor-core path");
    if (status != 0) {
        set_error("psf tensor-core path: a bounded wait for the tensor cores timed out");
        return FFT_ERR_TIMEOUT;
    }
    return FFT_OK;
}

}  // namespace fftgb
