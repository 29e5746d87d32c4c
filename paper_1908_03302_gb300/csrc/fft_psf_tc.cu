// Batched Hessian point-spread functions on the tensor cores (Sec. II-D, Eq. resolution_2):
//
//   Y[v, (s, k)] = sum_{p in S_s} J[p, v] J[p, spike_k]
//
// i.e. Y = J^T D with many right-hand sides, a dense contraction per voxel block: for an
// 8 x 4 x 4 sub-brick (128 voxels = the MMA's M) the rows whose support reaches it are the
// contraction dimension K and the spikes are N.
//
// Rows are grouped by the set of subsets that hold them (for nested ring subsets: the
// smallest subset holding the row). Group g accumulates Z_g[v, k] = sum_{p in g} J[p, v]
// J[p, spike_k] in its own block of TMEM columns, so every row carries one D entry per spike
// instead of one per (subset, spike), and a K chunk of one group multiplies only that group's
// columns. The epilogue forms Y[., (s, k)] = sum of Z_g over the groups whose rows belong to S_s
// (for nested subsets: prefix sums).
//
// One persistent CTA per SM runs a pipeline of three warp roles over units (tile, sub-brick):
//   * 3 scan warps stream the tile's compact candidate lists (built once per call by
//     psf_mask_kernel, one segment per group: the tile's rows that have D entries, each with its
//     staging record and the 16-bit mask of the sub-bricks its support may reach), keep the
//     rows whose mask holds the unit's sub-brick, 32 candidates per warp and block, and append
//     their records to a ring of 6 chunks of 96 rows in shared memory, groups in order and
//     candidates in order within a group (the blocks take turns), so the K order is fixed.
//     A chunk holds the rows of one group; it is published with a header (unit, rows, group,
//     first of the unit / of its group in the unit, last of the unit) on its "ring full"
//     mbarrier;
//   * 24 generator warps take the chunks in order: warp w covers 8 rows and 64 voxels; lane l
//     evaluates two rows on the 8 voxels of one x line of the sub-brick (FP32 evaluation as in
//     the J^T kernel, rounded to BF16) and writes them as eight 32-bit K pairs; the warp also
//     scatters the D entries (BF16, premultiplied by the row constant C_p) of 4 rows into the
//     chunk's B tile, then arrives on the stage's "full" mbarrier. After the last chunk of a
//     unit they move the accumulators TMEM -> registers -> Y and arrive on "TMEM free";
//   * 1 MMA warp waits for "full", issues tcgen05.mma (M = 128, N = the spikes of the block
//     rounded up to 16, K = 96 per chunk) into the chunk's group columns (the group's first
//     chunk of the unit starts a new accumulation; the unit's first waits for "TMEM free") and
//     commits to the stage's "done" mbarrier; one chunk later it waits for those MMAs and
//     zero-fills the stage's B tile with one bulk asynchronous copy from a zero page, which
//     completes the stage's "empty" mbarrier that the generators wait for before reusing it.
// Three A / B stages and the 6-chunk row ring decouple the roles: no CTA-wide barrier between
// the first and the last unit. The Phi tables are held in shared memory; where the geometry's
// tables and the stages do not fit together, the kernel takes the tables at half resolution
// (resampled from the device tables by the linear interpolant; the extra interpolation error,
// ~2e-5 of max |Phi|, is far below the BF16 rounding of the entries). Every wait is bounded; a
// thread whose wait timed out sets a status word and leaves its loop, so that the others time
// out in turn and the CTA ends.
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

constexpr int KC = 96;                 // rows per chunk (MMA K per chunk)
constexpr int GEN_WARPS = 24;          // warps that generate J and scatter D (warps 0 ..)
constexpr int ROW_OCTETS = KC / 8;     // generator warp w: rows 8 (w % 12) .., voxel half w / 12
constexpr int D_ROWS = KC / GEN_WARPS; // rows whose D entries a generator warp scatters
constexpr int SCAN_WARPS = 3;          // warps that scan candidate rows (warps 24 .. 26)
constexpr int MMA_WARP = GEN_WARPS + SCAN_WARPS;   // the warp that issues the MMAs
constexpr int TC_WARPS = MMA_WARP + 1;
constexpr int TC_THREADS = TC_WARPS * 32;
constexpr int NSTAGE = 3;              // A / B stages
constexpr int RING = 6;                // chunks of staged rows between the scan and the generation
constexpr int D_LANES = 16;            // lanes that scatter one row's D entries
constexpr long long WAIT_BUDGET = 4000000000ll;   // cycles (~2 s)
constexpr int HDR_UFIRST = 1, HDR_LAST = 2, HDR_GFIRST = 4;   // chunk header flags
constexpr int MAX_NG = 256;            // MMA N (spikes of one launch, rounded up to 16)
// Stand-in for a row past a chunk's end: a voxel line at distance FAR from the pair's axis and
// at its midplane (in band units), so that every detour form gives v = 2 FAR, saturated to the
// cut-off: Phi = 0, and the geometric factor stays finite.
constexpr float FAR = 1.0e4f;
static_assert(GEN_WARPS == 2 * ROW_OCTETS && D_ROWS == 4, "generator warps: 8 rows x 64 voxels");

// Zero page the MMA warp copies over a consumed B tile (static storage: zero-initialised).
__device__ __align__(128) uint4 g_zero_b[MAX_NG * KC * 2 / 16];

struct PsfTcParams {
    const RowRec* rec;
    const int32_t* row_band;
    const BandConst* bc;
    const float2* tab;
    int n_bands, n_tab;
    const int32_t* tile_rows;
    const int64_t* tile_off;
    const int32_t* tile_order;  // the pre-passes' CTA -> tile, heaviest tiles first
    const float4* ebase;
    const float* ebase3;
    const uint8_t* grp;        // group of each row (0xFF: the row is in no subset)
    int n_groups;              // G (<= PSF_TC_MAX_GROUPS)
    const int64_t* seg_off;    // [n_tiles * G] first compact candidate of (tile, group)
    float4* c_rec;             // compact candidates: staging record (3 float4, see psf_mask_kernel)
    int32_t* c_cnt;            // [n_tiles * G] compact candidates of (tile, group)
    const int32_t* units;      // (tile << 4) | sub-brick, heaviest tiles first
    int n_units;
    int32_t* counter;
    int tiles_x, tiles_y;
    int nx, ny, nz;
    const int64_t* d_off;      // sparse D rows: [M + 1]
    const uint32_t* d_ent;     // entry: spike index k (bits 0-15) | BF16 of C_p J[p, spike_k] (16-31)
    int ng;                    // MMA N: columns of one group (multiple of 16, <= MAX_NG)
    int tmem_cols;
    uint32_t gmask[PSF_TC_MAX_GROUPS];   // subsets that hold the rows of each group
    int n_sub;                 // subsets
    int n_spike, k0, nk;       // spikes of the call, first spike and spikes of this launch
    float* out;                // Y as out[(s * n_spike + k) * V + v]
    int64_t V;
    int32_t* status;
    unsigned long long* chunks;
};

struct ChunkHdr {
    int unit;     // (tile << 4) | sub-brick; n_rows < 0 ends the CTA's work
    int n_rows;   // staged rows in the chunk (0 .. KC)
    int flags;    // HDR_UFIRST, HDR_GFIRST, HDR_LAST
    int group;    // group of its rows
};

struct TcShared {
    unsigned long long full[NSTAGE];       // generator warps -> MMA warp (GEN_WARPS arrivals)
    unsigned long long done[NSTAGE];       // tensor cores -> MMA warp and epilogue (tcgen05.commit)
    unsigned long long empty[NSTAGE];      // MMA warp -> generator warps (B tile zero-filled: 1 arrival + bytes)
    unsigned long long ring_full[RING];    // scan warps -> generator and MMA warps (1 arrival)
    unsigned long long ring_empty[RING];   // generator and MMA warps -> scan warps (GEN_WARPS + 1)
    unsigned long long tmem_free;          // epilogue read the accumulators -> MMA warp (GEN_WARPS)
    unsigned long long unit_done;          // scan warps finished a unit (SCAN_WARPS arrivals)
    unsigned long long unit_ready;         // scan warp 0 fetched the next unit (1 arrival)
    ChunkHdr hdr[RING];
    BandConst bc[MAX_BANDS];
    uint32_t tmem_slot;
    int scan_unit;                         // unit index being scanned (>= n_units: no more)
    int turn;                              // next block of 32 candidates allowed to append
    int p_chunk;                           // producer: global index of the chunk being filled
    int p_fill;                            // its staged rows
    int p_flags;                           // its HDR_UFIRST / HDR_GFIRST flags
    int p_group;                           // its group (-1: none yet in this unit)
    int p_started;                         // the current unit has staged rows
};

// Bounded wait for a phase. Each poll lets the hardware suspend the thread for up to
// WAIT_HINT_NS while the phase is incomplete, so that waiting warps leave the issue slots to
// the generating ones.
constexpr uint32_t WAIT_HINT_NS = 1000;
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait_sleep(mbar, parity, WAIT_HINT_NS)) {
        if (clock64() - t0 > WAIT_BUDGET) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ void st_volatile(int* p, int v) { *reinterpret_cast<volatile int*>(p) = v; }

// Every lane of the warp waits (bounded) for the phase of `mbar` with the given parity, so each
// one acquires what the arrivals released. Returns false, for the whole warp, if some lane's
// wait timed out (status set).
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, int32_t* status) {
    const bool ok = wait_phase(mbar, parity);
    if (!ok) atomicExch(status, FFT_ERR_TIMEOUT);
    return __all_sync(0xffffffffu, ok);
}

// Producer side, called by the scan warp that holds the turn (whole warp): publish chunk
// `chunk` (lane 0 writes the header and arrives on its "ring full" barrier). The rows past
// n_rows get the stand-in record (a voxel line FAR from the pair's axis, no D entries, table
// base `tb_safe` with both detour-form flags), so that the generators load every row of a
// chunk alike and the stand-ins contribute exact zeros.
__device__ __forceinline__ void publish_chunk(TcShared& S, float4* s_ring, uint32_t ring_full0, int chunk, int unit,
                                              int n_rows, int flags, int group, uint32_t tb_safe, int lane) {
    if (n_rows >= 0) {
        float4* dst = s_ring + (size_t)(chunk % RING) * KC * 3;
        for (int r = n_rows + lane; r < KC; r += 32) {
            dst[3 * r + 0] = make_float4(0.f, 0.f, FAR, 0.f);
            dst[3 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            dst[3 * r + 2] = make_float4(0.f, __uint_as_float(tb_safe), 0.f, 0.f);
        }
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) {
        ChunkHdr& h = S.hdr[chunk % RING];
        h.unit = unit;
        h.n_rows = n_rows;
        h.flags = flags;
        h.group = group;
        tc::mbar_arrive(ring_full0 + 8u * (uint32_t)(chunk % RING));
    }
    __syncwarp();
}

// Before the first row of chunk `chunk` is staged, its ring slot must have been released by
// the consumers of chunk - RING.
__device__ __forceinline__ bool ring_slot_free(uint32_t ring_empty0, int chunk, int32_t* status) {
    if (chunk < RING) return true;
    return warp_wait(ring_empty0 + 8u * (uint32_t)(chunk % RING), (uint32_t)(((chunk / RING) - 1) & 1), status);
}

constexpr int MASK_THREADS = 256;

// Capacity of each (tile, group) candidate segment: the tile's entries whose row has D
// entries, by the row's group (an upper bound of the compact candidates psf_mask_kernel keeps).
__global__ void __launch_bounds__(MASK_THREADS) psf_cap_kernel(const PsfTcParams P, int32_t* __restrict__ cap) {
    __shared__ int s_cnt[PSF_TC_MAX_GROUPS];
    const int T = P.tile_order[blockIdx.x], G = P.n_groups;
    if (threadIdx.x < PSF_TC_MAX_GROUPS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t e = P.tile_off[T] + threadIdx.x; e < P.tile_off[T + 1]; e += MASK_THREADS) {
        const int p = P.tile_rows[e];
        if (P.d_off[p + 1] > P.d_off[p]) atomicAdd(&s_cnt[P.grp[p]], 1);
    }
    __syncthreads();
    if (threadIdx.x < G) cap[(int64_t)T * G + threadIdx.x] = s_cnt[threadIdx.x];
}

// Compact candidate lists, one CTA per tile: the tile's candidate rows that have D entries,
// each with the mask of its 16 sub-bricks (8 x 4 x 4, inside the grid) that the row's support
// may reach (tangent-plane bound of the convex detour, as in the J^T kernel), written by group
// from seg_off[T * G + g] in candidate order; c_cnt[T * G + g] their number and c_or[T] the
// union of the masks. With each candidate goes its staging record, so that the scan warps
// gather one contiguous record per kept row instead of chasing the entry, the row and its D
// offsets:
//   r0 = the entry's tile-origin base (p + L/2, p - L/2, c1, c2) in the pair frame,
//   r1 = (h e_x, h e_y, h e_z, c3) (pair-frame steps per voxel and the base's c3),
//   r2 = (mask of the sub-bricks, band index, first D entry of the row, D entries of the row)
//        (bits).
__global__ void __launch_bounds__(MASK_THREADS) psf_mask_kernel(const PsfTcParams P, uint16_t* __restrict__ c_or) {
    __shared__ int wsum[PSF_TC_MAX_GROUPS][MASK_THREADS / 32];
    __shared__ int64_t run[PSF_TC_MAX_GROUPS];
    __shared__ unsigned int s_or;
    const int T = P.tile_order[blockIdx.x], G = P.n_groups;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = T % P.tiles_x, ty = (T / P.tiles_x) % P.tiles_y, tz = T / (P.tiles_x * P.tiles_y);
    const int64_t e_begin = P.tile_off[T], e_end = P.tile_off[T + 1];
    if (threadIdx.x == 0) s_or = 0u;
    if (threadIdx.x < PSF_TC_MAX_GROUPS) run[threadIdx.x] = 0;
    __syncthreads();
    unsigned int my_or = 0u;
    for (int64_t e0 = e_begin; e0 < e_end; e0 += MASK_THREADS) {
        const int64_t e = e0 + threadIdx.x;
        unsigned int mask = 0u;
        int mg = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        if (e < e_end) {
            const int p = P.tile_rows[e];
            const int64_t d0 = P.d_off[p], d1 = P.d_off[p + 1];
            if (d1 > d0) {   // rows without D entries add nothing
                mg = P.grp[p];
                const RowRec r = P.rec[p];
                const int bnd = P.row_band[p];
                const BandConst bc = P.bc[bnd];
                const float hb = bc.h;
                r0 = P.ebase[e];
                r1 = make_float4(hb * r.b.x, hb * r.b.y, hb * r.b.z, P.ebase3[e]);
                r2 = make_float4(0.0f, __int_as_float(bnd), __uint_as_float((uint32_t)d0),
                                 __int_as_float((int)(d1 - d0)));
                for (int sb = 0; sb < 16; ++sb) {
                    const int X0 = TILE_X * tx + 8 * (sb & 1), Y0 = TILE_Y * ty + 4 * ((sb >> 1) & 3),
                              Z0 = TILE_Z * tz + 4 * (sb >> 3);
                    if (X0 >= P.nx || Y0 >= P.ny || Z0 >= P.nz) continue;
                    const float cx = fmaf((float)(X0) + 3.5f, hb, bc.org[0]) - r.a.x;
                    const float cy = fmaf((float)(Y0) + 1.5f, hb, bc.org[1]) - r.a.y;
                    const float cz = fmaf((float)(Z0) + 1.5f, hb, bc.org[2]) - r.a.z;
                    if (box_may_touch(cx, cy, cz, r.b.x, r.b.y, r.b.z, r.a.w, 3.5f * hb, 1.5f * hb, 1.5f * hb))
                        mask |= 1u << sb;
                }
            }
        }
        my_or |= mask;
        const bool keep = mask != 0u;
        // rank of this candidate among the block's kept candidates of its group
        int rank = 0;
        for (int g = 0; g < G; ++g) {
            const uint32_t bal = __ballot_sync(0xffffffffu, keep && mg == g);
            if (lane == 0) wsum[g][warp] = __popc(bal);
            if (keep && mg == g) rank = __popc(bal & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (keep) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += wsum[mg][w];
            const int64_t pos = P.seg_off[(int64_t)T * G + mg] + run[mg] + before + rank;
            P.c_rec[3 * pos + 0] = r0;
            P.c_rec[3 * pos + 1] = r1;
            r2.x = __uint_as_float(mask);
            P.c_rec[3 * pos + 2] = r2;
        }
        __syncthreads();
        if (threadIdx.x < G) {
            int total = 0;
            for (int w = 0; w < MASK_THREADS / 32; ++w) total += wsum[threadIdx.x][w];
            run[threadIdx.x] += total;
        }
        __syncthreads();
    }
    atomicOr(&s_or, my_or);
    __syncthreads();
    if (threadIdx.x < G) P.c_cnt[(int64_t)T * G + threadIdx.x] = (int32_t)run[threadIdx.x];
    if (threadIdx.x == 0) c_or[T] = (uint16_t)s_or;
}

// GUARD: some voxel centre lies on a transducer (the geometry's flag): the guarded detour.
template <bool GUARD>
__global__ void __launch_bounds__(TC_THREADS, 1) psf_tc_kernel(const __grid_constant__ PsfTcParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcShared S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- shared-memory carve-up: A[NSTAGE], B[NSTAGE] (1 KB aligned), tables, row ring
    const uint32_t a_bytes = 128u * KC * 2u;
    const uint32_t b_bytes = (uint32_t)P.ng * KC * 2u;
    unsigned char* sA0 = smem;
    unsigned char* sB0 = smem + NSTAGE * a_bytes;
    size_t off = NSTAGE * (size_t)a_bytes + NSTAGE * (size_t)b_bytes;
    float2* s_tab = reinterpret_cast<float2*>(smem + off);
    off += ((size_t)P.n_bands * P.n_tab * sizeof(float2) + 15) & ~(size_t)15;
    float4* s_ring = reinterpret_cast<float4*>(smem + off);   // [RING][KC][3] staged rows

    for (int i = tid; i < P.n_bands * P.n_tab; i += TC_THREADS) s_tab[i] = P.tab[i];
    if (tid < P.n_bands) S.bc[tid] = P.bc[tid];
    {   // B stages start cleared; afterwards the MMA warp zero-fills each one after its MMAs
        uint4* b4 = reinterpret_cast<uint4*>(sB0);
        for (uint32_t i = tid; i < NSTAGE * b_bytes / 16; i += TC_THREADS) b4[i] = make_uint4(0, 0, 0, 0);
    }
    const uint32_t tab_addr = smem_addr(s_tab);
    const uint32_t tb_safe = (tab_addr - MAGIC_BITS_X8) | 3u;   // band 0, both detour-form flags
    const float nm1 = (float)(P.n_tab - 1);
    const uint32_t full0 = smem_addr(&S.full[0]), empty0 = smem_addr(&S.empty[0]), done0 = smem_addr(&S.done[0]);
    const uint32_t ring_full0 = smem_addr(&S.ring_full[0]), ring_empty0 = smem_addr(&S.ring_empty[0]);
    const uint32_t tmem_free = smem_addr(&S.tmem_free);
    const uint32_t unit_done = smem_addr(&S.unit_done), unit_ready = smem_addr(&S.unit_ready);
    const int G = P.n_groups;
    if (warp == 0) {
        tc::tmem_alloc(smem_addr(&S.tmem_slot), (uint32_t)P.tmem_cols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < NSTAGE; ++b) {
            tc::mbar_init(full0 + 8u * b, GEN_WARPS);
            tc::mbar_init(done0 + 8u * b, 1);
            tc::mbar_init(empty0 + 8u * b, 1);
        }
        for (int b = 0; b < RING; ++b) {
            tc::mbar_init(ring_full0 + 8u * b, 1);
            tc::mbar_init(ring_empty0 + 8u * b, GEN_WARPS + 1);
        }
        tc::mbar_init(tmem_free, GEN_WARPS);
        tc::mbar_init(unit_done, SCAN_WARPS);
        tc::mbar_init(unit_ready, 1);
        S.p_chunk = 0;
        S.p_fill = 0;
        S.p_flags = HDR_UFIRST;
        S.p_group = -1;
        S.p_started = 0;
        S.turn = 0;
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();   // the only CTA-wide barrier before the teardown
    tc::fence_after_sync();
    const uint32_t taddr = S.tmem_slot;
    bool failed = false;
    int chunk = 0;   // chunks this warp has consumed (generator and MMA warps)

    if (warp >= GEN_WARPS && warp < MMA_WARP) {
        // ================= scan warps: candidate rows -> staged records in the row ring
        const int k = warp - GEN_WARPS;
        for (int u = 0;; ++u) {
            if (k == 0) {
                if (u > 0) {
                    // every scan warp has appended its blocks of the previous unit: close it
                    failed = failed || !warp_wait(unit_done, (uint32_t)((u - 1) & 1), P.status);
                    __threadfence_block();
                    if (!failed && S.p_started) {
                        const int pc = S.p_chunk, pf = S.p_fill;
                        // a unit whose rows filled its last chunk exactly gets an empty closing chunk
                        if (pf == 0) failed = failed || !ring_slot_free(ring_empty0, pc, P.status);
                        if (!failed)
                            publish_chunk(S, s_ring, ring_full0, pc, P.units[S.scan_unit], pf,
                                          HDR_LAST | S.p_flags, S.p_group, tb_safe, lane);
                        __syncwarp();
                        if (lane == 0) {
                            S.p_chunk = pc + 1;
                            S.p_fill = 0;
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    S.scan_unit = failed ? P.n_units : atomicAdd(P.counter, 1);
                    S.turn = 0;
                    S.p_flags = HDR_UFIRST;
                    S.p_group = -1;
                    S.p_started = 0;
                    __threadfence_block();
                    tc::mbar_arrive(unit_ready);
                }
                __syncwarp();
            } else {
                failed = failed || !warp_wait(unit_ready, (uint32_t)(u & 1), P.status);
            }
            __threadfence_block();
            const int unit = failed ? P.n_units : S.scan_unit;
            if (unit >= P.n_units) break;
            const int ucode = P.units[unit];
            const int T = ucode >> 4, sb = ucode & 15;
            const int tx = T % P.tiles_x, ty = (T / P.tiles_x) % P.tiles_y, tz = T / (P.tiles_x * P.tiles_y);
            const int X0 = TILE_X * tx + 8 * (sb & 1), Y0 = TILE_Y * ty + 4 * ((sb >> 1) & 3),
                      Z0 = TILE_Z * tz + 4 * (sb >> 3);
            const bool inside = X0 < P.nx && Y0 < P.ny && Z0 < P.nz;
            const int SXo = 8 * (sb & 1), SYo = 4 * ((sb >> 1) & 3), SZo = 4 * (sb >> 3);   // in the tile
            // the tile's groups: lane g holds group g's candidate count, first candidate and
            // (inclusive prefix) the end of its blocks of 32 in the unit's block sequence
            int g_cnt = 0;
            long long g_seg = 0;
            if (inside && lane < G) {
                g_cnt = P.c_cnt[(int64_t)T * G + lane];
                g_seg = P.seg_off[(int64_t)T * G + lane];
            }
            const int g_nb = (g_cnt + 31) >> 5;
            int g_end = g_nb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, g_end, o);
                if (lane >= o) g_end += x;
            }
            const int n_blocks = __shfl_sync(0xffffffffu, g_end, 31);
            // the gathers of block b (its group g, its block bl within the group): the staging
            // record of each lane's candidate (its sub-brick mask in r2.x), zero past the group's end
            auto gather = [&](int b, float4& r0, float4& r1, float4& r2) {
                r0 = r1 = r2 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (b >= n_blocks) return;
                const int g = __popc(__ballot_sync(0xffffffffu, g_end <= b));
                const int bl = b - (__shfl_sync(0xffffffffu, g_end, g) - __shfl_sync(0xffffffffu, g_nb, g));
                const int n_c = __shfl_sync(0xffffffffu, g_cnt, g);
                const long long seg = __shfl_sync(0xffffffffu, g_seg, g);
                const int ci = 32 * bl + lane;
                if (ci < n_c) {
                    const int64_t c = seg + ci;
                    r0 = P.c_rec[3 * c + 0];
                    r1 = P.c_rec[3 * c + 1];
                    r2 = P.c_rec[3 * c + 2];
                }
            };
            for (int b = k; b < n_blocks && !failed; b += SCAN_WARPS) {
                float4 s0, s1, s2;
                gather(b, s0, s1, s2);
                const int g = __popc(__ballot_sync(0xffffffffu, g_end <= b));
                // ---- block b: keep the candidates that reach the sub-brick
                const bool keep = (__float_as_uint(s2.x) >> sb) & 1u;
                if (keep) {
                    // is the whole sub-brick between the transducer planes (|p| <= L / 2 at every
                    // voxel centre)? p at its centre from the tile-origin base and the steps
                    const float hx = s1.x, hy = s1.y, hz = s1.z;
                    const float p0 = 0.5f * (s0.x + s0.y), hl = 0.5f * (s0.x - s0.y);
                    const float pc = fmaf((float)(SXo + 3.5f), hx, fmaf((float)(SYo + 1.5f), hy, fmaf((float)(SZo + 1.5f), hz, p0)));
                    const float pext = 3.5f * fabsf(hx) + 1.5f * (fabsf(hy) + fabsf(hz)) + 1e-3f;
                    const bool inner = fabsf(pc) + pext <= hl;
                    // table base (a multiple of 8) with the inner / planar flags in bits 0, 1
                    const uint32_t bnd = (uint32_t)__float_as_int(s2.y);
                    const uint32_t tb = (tab_addr + bnd * (uint32_t)P.n_tab * 8u - MAGIC_BITS_X8) | (inner ? 1u : 0u) |
                                        (hz == 0.0f ? 2u : 0u);
                    s2.y = __uint_as_float(tb);
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                // ---- wait for this block's turn, then append its kept rows in lane order
                bool ok = true;
                {   // back off while waiting, so that the spin does not take issue slots from the
                    // generator warps on this SM sub-partition
                    const long long t0 = clock64();
                    while (ld_volatile(&S.turn) != b) {
                        __nanosleep(64);
                        if (clock64() - t0 > WAIT_BUDGET) {
                            atomicExch(P.status, FFT_ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
                failed = failed || !__all_sync(0xffffffffu, ok);
                if (failed) break;
                __threadfence_block();
                const int n = __popc(bal);
                if (n > 0) {
                    int pc = S.p_chunk, pf = S.p_fill, fl = S.p_flags, cg = S.p_group;
                    if (cg != g) {   // a chunk holds one group: close the other group's chunk
                        if (pf > 0) {
                            publish_chunk(S, s_ring, ring_full0, pc, ucode, pf, fl, cg, tb_safe, lane);
                            ++pc;
                            pf = 0;
                            fl &= ~HDR_UFIRST;
                        }
                        cg = g;
                        fl |= HDR_GFIRST;
                    }
                    // the slots the rows go to must be free: the current chunk's (if it starts
                    // here) and the next one's (if the rows spill over)
                    if (pf == 0) failed = failed || !ring_slot_free(ring_empty0, pc, P.status);
                    if (pf + n > KC) failed = failed || !ring_slot_free(ring_empty0, pc + 1, P.status);
                    if (failed) break;
                    if (keep) {
                        const int pos = pf + __popc(bal & ((1u << lane) - 1u));
                        const int cc = pc + pos / KC, rr = pos % KC;
                        float4* dst = s_ring + ((size_t)(cc % RING) * KC + rr) * 3;
                        dst[0] = s0;
                        dst[1] = s1;
                        dst[2] = s2;
                    }
                    int nf = pf + n;
                    if (nf >= KC) {   // the chunk is full: publish it
                        publish_chunk(S, s_ring, ring_full0, pc, ucode, KC, fl, cg, tb_safe, lane);
                        ++pc;
                        nf -= KC;
                        fl = 0;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        S.p_chunk = pc;
                        S.p_fill = nf;
                        S.p_flags = fl;
                        S.p_group = cg;
                        S.p_started = 1;
                    }
                }
                __threadfence_block();
                __syncwarp();
                if (lane == 0) st_volatile(&S.turn, b + 1);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(unit_done);
        }
        if (k == 0 && !failed) {   // no more units: tell the consumers
            const int pc = S.p_chunk;
            if (ring_slot_free(ring_empty0, pc, P.status))
                publish_chunk(S, s_ring, ring_full0, pc, 0, -1, 0, 0, tb_safe, lane);
        }
    } else if (warp < GEN_WARPS) {
        // ================= generator warps
        // Warp w covers rows 8 ro .. 8 ro + 7 of a chunk (ro = w % 12) and voxel half hv = w / 12
        // of the 8 x 4 x 4 sub-brick (z layers 2 hv, 2 hv + 1). Lane l evaluates rows
        // 8 ro + 2 rp and 8 ro + 2 rp + 1 (rp = l >> 3) on the x line (t = 0 .. 7, g & 3,
        // 2 hv + (g >> 2)) of the sub-brick, g = l & 7. Voxel t of lane l is MMA row (TMEM lane)
        // m = 64 hv + 8 t + g: one store instruction then writes eight rows m and four K pairs of
        // one core matrix, 32 distinct banks. For D the warp owns B-tile rows 4 w .. 4 w + 3 of
        // every stage, two at a time (lanes 0-15 and 16-31); lane i of a half scatters the row's
        // D entries i, i + 16, i + 32, ...
        const int ro = warp % ROW_OCTETS, hv = warp / ROW_OCTETS;
        const int rp = lane >> 3, gg = lane & 7;
        const int ra = 8 * ro + 2 * rp;   // this lane's rows ra, ra + 1
        const int d_i0 = lane & (D_LANES - 1);
        // byte offset of (MMA row 64 hv + g, K pair ra) in a stage; voxel t adds t x 16 KC
        const uint32_t a_off0 = tc::kmajor_offset((uint32_t)(64 * hv + gg), (uint32_t)ra, KC);
        const float Yv0 = (float)(gg & 3), Zv0 = (float)(2 * hv + (gg >> 2));
        uint32_t upres = 0u;   // groups with chunks in the current unit
        for (;; ++chunk) {
            const int slot = chunk % RING;
            if (!warp_wait(ring_full0 + 8u * slot, (uint32_t)((chunk / RING) & 1), P.status)) {
                failed = true;
                break;
            }
            const ChunkHdr h = S.hdr[slot];
            if (h.n_rows < 0) break;
            upres |= 1u << h.group;
            const int T = h.unit >> 4, sb = h.unit & 15;
            const int SX = 8 * (sb & 1), SY = 4 * ((sb >> 1) & 3), SZ = 4 * (sb >> 3);
            const float4* stg = s_ring + (size_t)slot * KC * 3;
            const int buf = chunk % NSTAGE;
            const uint32_t use = (uint32_t)(chunk / NSTAGE);
            unsigned char* sA = sA0 + buf * a_bytes;
            unsigned char* sB = sB0 + buf * b_bytes;
            // D entries of this warp's B rows 4 w + 2 dp + (lane >> 4): loads issued now, stored
            // after the generation
            int d_cnt[2];
            uint32_t d_beg[2], e0[2], e1[2];
#pragma unroll
            for (int dp = 0; dp < 2; ++dp) {
                const int dr = D_ROWS * warp + 2 * dp + (lane >> 4);
                const float4 C = stg[dr * 3 + 2];   // a stand-in row has no D entries
                d_beg[dp] = __float_as_uint(C.z);
                d_cnt[dp] = __float_as_int(C.w);
                e0[dp] = d_i0 < d_cnt[dp] ? P.d_ent[d_beg[dp] + d_i0] : 0u;
                e1[dp] = d_i0 + D_LANES < d_cnt[dp] ? P.d_ent[d_beg[dp] + d_i0 + D_LANES] : 0u;
            }
            // the MMAs that last read this stage must be done and its B tile cleared
            if (chunk >= NSTAGE && !warp_wait(empty0 + 8u * buf, (use - 1u) & 1u, P.status)) {
                failed = true;
                break;
            }
            // generate A: this lane's rows ra, ra + 1 on its eight voxels (a row past the chunk's
            // end is the producer's stand-in: Phi = 0 exactly). The detour form is chosen per
            // warp: the inner / planar forms only where all its rows allow them.
            const float4 Aa = stg[ra * 3 + 0], Ba = stg[ra * 3 + 1];
            const uint32_t ta = __float_as_uint(stg[ra * 3 + 2].y);
            const float4 Ab = stg[ra * 3 + 3], Bb = stg[ra * 3 + 4];
            const uint32_t tbb = __float_as_uint(stg[ra * 3 + 5].y);
            const uint32_t fl = ta & tbb & 3u;
            const uint32_t wfl = (__all_sync(0xffffffffu, fl & 1u) ? 1u : 0u) | (__all_sync(0xffffffffu, fl & 2u) ? 2u : 0u);
            const float Xv = (float)SX, Yv = (float)SY + Yv0, Zv = (float)SZ + Zv0;
            // pair-frame values of each row at voxel t = 0 of the lane's line
            const float oa = fmaf(Xv, Ba.x, fmaf(Yv, Ba.y, Zv * Ba.z)), ob = fmaf(Xv, Bb.x, fmaf(Yv, Bb.y, Zv * Bb.z));
            const float psa = Aa.x + oa, pra = Aa.y + oa, psb = Ab.x + ob, prb = Ab.y + ob;
            const float c1a = fmaf(Yv, Ba.z, fmaf(-Zv, Ba.y, Aa.z)), c1b = fmaf(Yv, Bb.z, fmaf(-Zv, Bb.y, Ab.z));
            const float c2a = fmaf(Zv, Ba.x, fmaf(-Xv, Ba.z, Aa.w)), c2b = fmaf(Zv, Bb.x, fmaf(-Xv, Bb.z, Ab.w));
            const float c3a = fmaf(Xv, Ba.y, fmaf(-Yv, Ba.x, Ba.w)), c3b = fmaf(Xv, Bb.y, fmaf(-Yv, Bb.x, Bb.w));
            const float c1qa = c1a * c1a, c1qb = c1b * c1b;
            const float c12a = fmaf(c2a, c2a, c1qa), c12b = fmaf(c2b, c2b, c1qb);
            const uint32_t tba = ta & ~3u, tbbb = tbb & ~3u;
            unsigned char* aw = sA + a_off0;
            // warp-uniform choice of the detour form for the whole line
#define FFT_TC_LINE(INNER_V, PLANAR_V)                                                                 \
    _Pragma("unroll") for (int t = 0; t < 8; ++t) {                                                   \
        const float ft = (float)t;                                                                    \
        float q2a, q2b;                                                                               \
        const float c3ta = fmaf(ft, Ba.y, c3a), c3tb = fmaf(ft, Bb.y, c3b);                           \
        if (PLANAR_V) {                                                                               \
            q2a = fmaf(c3ta, c3ta, c12a);                                                             \
            q2b = fmaf(c3tb, c3tb, c12b);                                                             \
        } else {                                                                                      \
            const float c2ta = fmaf(-ft, Ba.z, c2a), c2tb = fmaf(-ft, Bb.z, c2b);                     \
            q2a = fmaf(c2ta, c2ta, fmaf(c3ta, c3ta, c1qa));                                           \
            q2b = fmaf(c2tb, c2tb, fmaf(c3tb, c3tb, c1qb));                                           \
        }                                                                                             \
        float isa, ira, isb, irb;                                                                     \
        const float via = detour_v<FFT_DT_STABLE, GUARD, INNER_V>(fmaf(ft, Ba.x, psa), fmaf(ft, Ba.x, pra), q2a, \
                                                                 0.0f, isa, ira);                     \
        const float vib = detour_v<FFT_DT_STABLE, GUARD, INNER_V>(fmaf(ft, Bb.x, psb), fmaf(ft, Bb.x, prb), q2b, \
                                                                 0.0f, isb, irb);                     \
        const float ya = phi_lookup(via, tba, nm1) * (isa * ira);                                    \
        const float yb = phi_lookup(vib, tbbb, nm1) * (isb * irb);                                   \
        *reinterpret_cast<uint32_t*>(aw + t * 16 * KC) = pack_bf16x2(ya, yb);                        \
    }
            if (wfl & 1u) {
                if (wfl & 2u) {
                    FFT_TC_LINE(true, true)
                } else {
                    FFT_TC_LINE(true, false)
                }
            } else {
                if (wfl & 2u) {
                    FFT_TC_LINE(false, true)
                } else {
                    FFT_TC_LINE(false, false)
                }
            }
#undef FFT_TC_LINE
            // B: the stage was zero-filled (bulk copy issued by the MMA warp); scatter the rows'
            // D entries (BF16 of C_p J[p, spike_k] in bits 16-31, spike k in bits 0-15)
#pragma unroll
            for (int dp = 0; dp < 2; ++dp) {
                const uint32_t kr = (uint32_t)(D_ROWS * warp + 2 * dp + (lane >> 4));
                if (d_i0 < d_cnt[dp])
                    *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset(e0[dp] & 0xFFFFu, kr, KC)) =
                        (uint16_t)(e0[dp] >> 16);
                if (d_i0 + D_LANES < d_cnt[dp])
                    *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset(e1[dp] & 0xFFFFu, kr, KC)) =
                        (uint16_t)(e1[dp] >> 16);
                for (int i = d_i0 + 2 * D_LANES; i < d_cnt[dp]; i += D_LANES) {   // long rows
                    const uint32_t en = P.d_ent[d_beg[dp] + i];
                    *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset(en & 0xFFFFu, kr, KC)) = (uint16_t)(en >> 16);
                }
            }
            // publish this warp's part of the chunk to the MMA warp; release the ring slot
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(full0 + 8u * buf);
                tc::mbar_arrive(ring_empty0 + 8u * slot);
            }
            if (h.flags & HDR_LAST) {
                // ---- all MMAs of the unit done (they complete in order) -> TMEM -> Y
                if (!warp_wait(done0 + 8u * buf, use & 1u, P.status)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const int tx = T % P.tiles_x, ty = (T / P.tiles_x) % P.tiles_y, tz = T / (P.tiles_x * P.tiles_y);
                const int X0 = TILE_X * tx + SX, Y0 = TILE_Y * ty + SY, Z0 = TILE_Z * tz + SZ;
                const int quarter = warp & 3;   // TMEM lanes this warp may access
                // TMEM lane m = 32 quarter + lane holds voxel (t, g & 3, 2 hv + (g >> 2)) with
                // hv = quarter >> 1, t = 4 (quarter & 1) + (lane >> 3), g = lane & 7 (the
                // generators' row order)
                const int eg = lane & 7;
                const int x = X0 + 4 * (quarter & 1) + (lane >> 3), y = Y0 + (eg & 3),
                          z = Z0 + 2 * (quarter >> 1) + (eg >> 2);
                const bool valid = x < P.nx && y < P.ny && z < P.nz;
                const int64_t v = ((int64_t)z * P.ny + y) * P.nx + x;
                const uint32_t lane_base = taddr + ((uint32_t)(32 * quarter) << 16);
                for (int c = 8 * (warp >> 2); c < P.nk; c += 8 * (GEN_WARPS / 4)) {
                    for (int s = 0; s < P.n_sub; ++s) {
                        float acc[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) acc[i] = 0.0f;
                        for (int g = 0; g < G; ++g) {
                            if (!((upres >> g) & 1u) || !((P.gmask[g] >> s) & 1u)) continue;
                            float ov[8];
                            tc::tmem_ld_x8(lane_base + (uint32_t)(g * P.ng + c), ov);
#pragma unroll
                            for (int i = 0; i < 8; ++i) acc[i] += ov[i];
                        }
                        if (valid) {
                            float* o = P.out + ((int64_t)s * P.n_spike + P.k0 + c) * P.V + v;
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                if (c + i < P.nk) o[(int64_t)i * P.V] = acc[i];
                        }
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tmem_free);
                upres = 0u;
            }
        }
    } else {
        // ================= MMA warp
        const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)P.ng);
        int units = 0;    // units whose first chunk was issued
        int copied = 0;   // chunks whose B stage got its zero-fill copy (0 .. copied - 1)
        for (;; ++chunk) {
            const int slot = chunk % RING;
            if (!warp_wait(ring_full0 + 8u * slot, (uint32_t)((chunk / RING) & 1), P.status)) {
                failed = true;
                break;
            }
            const ChunkHdr h = S.hdr[slot];
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(ring_empty0 + 8u * slot);
            if (h.n_rows < 0) break;
            const bool ufirst = (h.flags & HDR_UFIRST) != 0, gfirst = (h.flags & HDR_GFIRST) != 0;
            // a new unit overwrites TMEM: the previous unit's epilogue must have read it
            if (ufirst && units > 0 && !warp_wait(tmem_free, (uint32_t)((units - 1) & 1), P.status)) {
                failed = true;
                break;
            }
            if (ufirst) ++units;
            const int buf = chunk % NSTAGE;
            const uint32_t use = (uint32_t)(chunk / NSTAGE);
            if (!warp_wait(full0 + 8u * buf, use & 1u, P.status)) {
                failed = true;
                break;
            }
            if (lane == 0) {
                tc::fence_after_sync();
                const uint32_t a_base = smem_addr(sA0 + buf * a_bytes), b_base = smem_addr(sB0 + buf * b_bytes);
                const uint32_t d_col = taddr + (uint32_t)(h.group * P.ng);
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    const uint64_t ad = tc::smem_desc(a_base + 256u * ks, 128u, 16u * KC);
                    const uint64_t bd = tc::smem_desc(b_base + 256u * ks, 128u, 16u * KC);
                    tc::mma_bf16(d_col, ad, bd, idesc, (!gfirst || ks > 0) ? 1u : 0u);
                }
                tc::mma_commit(done0 + 8u * buf);
            }
            __syncwarp();
            // the previous chunk's MMAs are done (they complete in order, before this chunk's):
            // zero its B tile with a bulk copy from a zero page in global memory, which
            // completes the stage's "empty" phase when its bytes have landed
            if (chunk > 0) {
                const int prev = chunk - 1;
                const int pbuf = prev % NSTAGE;
                if (!warp_wait(done0 + 8u * pbuf, (uint32_t)((prev / NSTAGE) & 1), P.status)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                if (lane == 0) {
                    tc::mbar_arrive_expect_tx(empty0 + 8u * pbuf, b_bytes);
                    tc::bulk_copy_g2s(smem_addr(sB0 + pbuf * b_bytes), g_zero_b, b_bytes, empty0 + 8u * pbuf);
                }
                copied = chunk;
                __syncwarp();
            }
        }
        // drain: every issued MMA must be complete before the accumulator is released
        if (chunk > 0) {   // MMAs complete in order: the last one done means all are done
            const int last = chunk - 1;
            if (lane == 0) wait_phase(done0 + 8u * (last % NSTAGE), (uint32_t)((last / NSTAGE) & 1));
            __syncwarp();
        }
        // and every zero-fill copy must have landed before the CTA's shared memory goes away:
        // the last copy into each stage is that stage's latest "empty" phase
        if (lane == 0)
            for (int c = copied > NSTAGE ? copied - NSTAGE : 0; c < copied; ++c)
                wait_phase(empty0 + 8u * (c % NSTAGE), (uint32_t)((c / NSTAGE) & 1));
        __syncwarp();
        if (lane == 0 && chunk > 0) atomicAdd(P.chunks, (unsigned long long)chunk);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tmem_cols);
}

}  // namespace

static size_t psf_tc_smem(fft_geom g, int ng, int n_tab) {
    return NSTAGE * (size_t)(128 * KC * 2) + NSTAGE * (size_t)ng * KC * 2 +
           (((size_t)g->n_bands * n_tab * sizeof(float2) + 15) & ~(size_t)15) +
           (size_t)RING * KC * 3 * sizeof(float4) + sizeof(TcShared) + 1024;
}

// Table length the tensor-core kernel uses: the geometry's, or half of it (n -> (n + 1) / 2
// samples) while all band tables take more than 48 KB of shared memory.
static int psf_tc_table_len(fft_geom g) {
    int n = g->n_tab;
    while (n > 64 && (size_t)g->n_bands * n * sizeof(float2) > 48 * 1024) n = (n + 1) / 2;
    return n;
}

// Band tables at n2 samples from the device tables at n samples (packed as (Phi_k - k dPhi_k,
// (n - 1) dPhi_k)): Phi at v = k / (n2 - 1) by the linear interpolant of the original, in FP64,
// packed the same way; the last entry is the cut-off (0, 0).
__global__ void psf_tc_resample_kernel(const float2* __restrict__ tab, int n, int n_bands, int n2,
                                       float2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_bands * n2) return;
    const int b = i / n2, k = i % n2;
    const float2* t = tab + (size_t)b * n;
    auto phi = [&](int kk) -> double {
        if (kk >= n2 - 1) return 0.0;
        const double v = (double)kk / (double)(n2 - 1);
        int j = (int)floor(v * (double)(n - 1));
        j = j < 0 ? 0 : (j > n - 2 ? n - 2 : j);
        return (double)t[j].x + v * (double)t[j].y;
    };
    if (k == n2 - 1) {
        out[i] = make_float2(0.0f, 0.0f);
    } else {
        const double p0 = phi(k), d = phi(k + 1) - p0;
        out[i] = make_float2((float)(p0 - (double)k * d), (float)(d * (double)(n2 - 1)));
    }
}

// Largest number of spikes one tensor-core launch can take with n_groups row groups on this
// device: the B stages grow with the spikes (rounded up to 16) and the accumulators take
// n_groups x that many TMEM columns (at most 512); 0 if even 16 do not fit.
int psf_tc_max_spikes(fft_geom g, int n_groups) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 0;
    for (int ng = 16; ng <= MAX_NG && n_groups * ng <= 512; ng += 16)
        if (psf_tc_smem(g, ng, psf_tc_table_len(g)) <= (size_t)optin) best = ng;
    return best;
}

// Y = J^T D on the tensor cores for one block of spikes: D given as sparse rows (d_off, d_ent:
// one entry per spike with J[p, spike] != 0, for the rows in some subset), the rows' groups
// (grp, and gmask[g] the subsets holding group g's rows). Writes out[(s * n_spike + k0 + k) * V
// + v] for k < nk; out must be zeroed by the caller (voxels that no row reaches are not
// written). Synchronous; returns FFT_ERR_TIMEOUT if a bounded wait gave up.
fft_status launch_psf_tc(fft_geom g, const int64_t* d_off, const uint32_t* d_ent, const uint8_t* grp, int n_groups,
                         const uint32_t* gmask, int n_sub, int n_spike, int k0, int nk, float* out, cudaStream_t st) {
    if (n_groups < 1 || n_groups > PSF_TC_MAX_GROUPS || nk < 1) {
        set_error("psf tensor-core path: 1 .. 32 row groups and at least one spike per launch");
        return FFT_ERR_ARG;
    }
    if (g->E == 0) return FFT_OK;
    const int ng = (int)ceil_div(nk, 16) * 16;
    if (ng > MAX_NG || n_groups * ng > 512) {
        set_error("psf tensor-core path: too many spikes for one launch");
        return FFT_ERR_ARG;
    }
    int tmem_cols = 32;
    while (tmem_cols < n_groups * ng) tmem_cols <<= 1;

    PsfTcParams P;
    memset(&P, 0, sizeof(P));
    P.rec = g->rec;
    P.row_band = g->row_band;
    P.bc = g->d_band;
    P.tab = g->tab;
    P.n_bands = g->n_bands;
    P.n_tab = g->n_tab;
    const int n_tab_tc = psf_tc_table_len(g);
    P.tile_rows = g->tile_rows;
    P.tile_off = g->tile_off;
    P.ebase = g->ebase;
    P.ebase3 = g->ebase3;
    P.grp = grp;
    P.n_groups = n_groups;
    P.tiles_x = g->tiles[0];
    P.tiles_y = g->tiles[1];
    P.nx = g->grid.nx;
    P.ny = g->grid.ny;
    P.nz = g->grid.nz;
    P.d_off = d_off;
    P.d_ent = d_ent;
    P.ng = ng;
    P.tmem_cols = tmem_cols;
    for (int i = 0; i < n_groups; ++i) P.gmask[i] = gmask[i];
    P.n_sub = n_sub;
    P.n_spike = n_spike;
    P.k0 = k0;
    P.nk = nk;
    P.out = out;
    P.V = g->V;

    // compact candidate lists by group (rows with D entries and their staging records, which
    // hold the sub-brick masks; 48 bytes per tile entry at most): segment capacities first, then the
    // lists, then the units: the sub-bricks that some candidate of their tile may reach,
    // heaviest tiles first
    const int64_t n_seg = g->n_tiles * n_groups;
    int32_t *c_cnt = nullptr, *d_units = nullptr, *d_ctr = nullptr, *d_cap = nullptr, *d_order = nullptr;
    int64_t* d_seg = nullptr;
    float4* c_rec = nullptr;
    uint16_t* c_or = nullptr;
    float2* tab_tc = nullptr;
    auto release = [&]() {   // (the candidate records stay with the geometry)
        cudaFree(tab_tc);
        cudaFree(c_cnt);
        cudaFree(c_or);
        cudaFree(d_units);
        cudaFree(d_ctr);
        cudaFree(d_cap);
        cudaFree(d_seg);
        cudaFree(d_order);
    };
    // the pre-passes run one CTA per tile; tiles differ in size by orders of magnitude, so
    // the heaviest start first and the small ones fill in behind them
    std::vector<int64_t> toff(g->n_tiles + 1);
    std::vector<int32_t> order(g->n_tiles);
    cudaError_t e = cudaMemcpy(toff.data(), g->tile_off, sizeof(int64_t) * toff.size(), cudaMemcpyDeviceToHost);
    for (int64_t T = 0; T < g->n_tiles; ++T) order[T] = (int32_t)T;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return toff[a + 1] - toff[a] > toff[b + 1] - toff[b]; });
    if (e == cudaSuccess) e = cudaMalloc(&d_order, sizeof(int32_t) * (size_t)g->n_tiles);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, st);
    P.tile_order = d_order;
    if (e == cudaSuccess) e = cudaMalloc(&d_cap, sizeof(int32_t) * (size_t)n_seg);
    if (e == cudaSuccess) e = cudaMalloc(&d_seg, sizeof(int64_t) * (size_t)n_seg);
    if (e == cudaSuccess) e = cudaMalloc(&c_cnt, sizeof(int32_t) * (size_t)n_seg);
    if (e == cudaSuccess) e = cudaMalloc(&c_or, sizeof(uint16_t) * (size_t)g->n_tiles);
    if (e == cudaSuccess) e = cudaMalloc(&d_ctr, 4 * sizeof(int32_t));   // counter, status, 64-bit chunk count
    if (e == cudaSuccess && n_tab_tc != g->n_tab) {
        e = cudaMalloc(&tab_tc, sizeof(float2) * (size_t)g->n_bands * n_tab_tc);
        if (e == cudaSuccess) {
            const int nt = g->n_bands * n_tab_tc;
            psf_tc_resample_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, st>>>(g->tab, g->n_tab, g->n_bands,
                                                                                n_tab_tc, tab_tc);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        psf_cap_kernel<<<(unsigned)g->n_tiles, MASK_THREADS, 0, st>>>(P, d_cap);
        e = cudaGetLastError();
    }
    std::vector<int32_t> cap(n_seg);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cap.data(), d_cap, sizeof(int32_t) * cap.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<int64_t> seg(n_seg);
    int64_t n_cand = 0;
    for (int64_t i = 0; i < n_seg; ++i) {
        seg[i] = n_cand;
        n_cand += cap[i];
    }
    if (e == cudaSuccess && n_cand == 0) {
        release();
        return FFT_OK;
    }
    // the candidate records (16 GB for psf3d) stay with the geometry and grow as needed:
    // allocating and freeing them took ~9 ms per call
    if (e == cudaSuccess && g->psf_crec_cap < n_cand) {
        cudaFree(g->psf_crec);
        g->scratch_bytes -= (int64_t)(3 * sizeof(float4)) * g->psf_crec_cap;
        g->psf_crec = nullptr;
        g->psf_crec_cap = 0;
        e = cudaMalloc(&g->psf_crec, 3 * sizeof(float4) * (size_t)n_cand);
        if (e == cudaSuccess) {
            g->psf_crec_cap = n_cand;
            g->scratch_bytes += (int64_t)(3 * sizeof(float4)) * n_cand;
        }
    }
    c_rec = g->psf_crec;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_seg, seg.data(), sizeof(int64_t) * seg.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "psf tensor-core path: candidate lists");
    }
    P.seg_off = d_seg;
    P.c_rec = c_rec;
    P.c_cnt = c_cnt;
    psf_mask_kernel<<<(unsigned)g->n_tiles, MASK_THREADS, 0, st>>>(P, c_or);
    e = cudaGetLastError();
    std::vector<int32_t> cnt(n_seg);
    std::vector<uint16_t> ors(g->n_tiles);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), c_cnt, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ors.data(), c_or, sizeof(uint16_t) * ors.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "psf tensor-core path: candidate lists");
    }
    std::vector<int64_t> tcount(g->n_tiles, 0);
    std::vector<int32_t> tiles;
    for (int64_t T = 0; T < g->n_tiles; ++T) {
        for (int gi = 0; gi < n_groups; ++gi) tcount[T] += cnt[T * n_groups + gi];
        if (tcount[T] > 0) tiles.push_back((int32_t)T);
    }
    std::stable_sort(tiles.begin(), tiles.end(), [&](int32_t a, int32_t b) { return tcount[a] > tcount[b]; });
    std::vector<int32_t> units;
    units.reserve(tiles.size() * 16);
    for (int32_t T : tiles)
        for (int s = 0; s < 16; ++s)
            if ((ors[T] >> s) & 1u) units.push_back((T << 4) | s);
    if (units.empty()) {
        release();
        return FFT_OK;
    }
    e = cudaMalloc(&d_units, sizeof(int32_t) * units.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_units, units.data(), sizeof(int32_t) * units.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, 4 * sizeof(int32_t), st);
    P.units = d_units;
    P.n_units = (int)units.size();
    P.counter = d_ctr;
    P.status = d_ctr + 1;
    P.chunks = reinterpret_cast<unsigned long long*>(d_ctr + 2);

    if (tab_tc) {   // the kernel's tables: the resampled ones
        P.tab = tab_tc;
        P.n_tab = n_tab_tc;
    }
    // at least 120 KB so that only one CTA (which holds TMEM for the whole launch) fits on an SM
    const size_t smem = std::max<size_t>(120 * 1024, psf_tc_smem(g, ng, n_tab_tc) - sizeof(TcShared) - 1024);
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && smem + sizeof(TcShared) > (size_t)optin) {
        release();
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
    // MMA work of this launch: every chunk multiplies a 128 x KC BF16 tile by KC x ng
    g->psf_tc_mma_flops += 2.0 * 128.0 * KC * (double)ng * (double)nch;
    g->psf_tc_entries += 128.0 * KC * (double)nch;
    release();
    if (e != cudaSuccess) return cuda_fail(e, "psf tensor-core path");
    if (status != 0) {
        set_error("psf tensor-core path: a bounded wait for the tensor cores timed out");
        return FFT_ERR_TIMEOUT;
    }
    return FFT_OK;
}

}  // namespace fftgb
