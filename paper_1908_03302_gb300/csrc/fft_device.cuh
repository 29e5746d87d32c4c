// Device-side building blocks of the J / J^T evaluation (Sec. II-C, Eq. Kernel_freq).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_common.cuh"

namespace fftgb {

// 1.5 * 2^23: adding it to a float in [0, 2^22) leaves the integer part in the low mantissa bits.
constexpr float MAGIC = 12582912.0f;
constexpr uint32_t MAGIC_BITS_X8 = 0x4B400000u << 3;   // wraps modulo 2^32 on purpose

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ float lds_f1(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Conservative test: may the row's support {R < 1} (band units) reach a box of voxel
// centres with centre c and half extents hx, hy, hz? R(x) = |x - xs| + |x - xr| - 2 hl is
// convex, so every tangent plane lies below it: R(x) >= R(x1) + grad R(x1) . (x - x1), whose
// minimum over the box is R(x1) + grad R(x1) . (c - x1) - sum_k |dR/dx_k(x1)| half_k. The box
// is culled when that minimum reaches 1 for the plane at the centre, or for a second plane
// at the corner where the centre's plane is lowest (which removes most of the boxes the first
// plane keeps without any in-support voxel centre). d = c - o is the centre relative to the
// pair midpoint, e the unit pair axis.
__device__ __forceinline__ float tangent_box_min(float x1x, float x1y, float x1z, float cx, float cy, float cz,
                                                 float ex, float ey, float ez, float hl, float hx, float hy,
                                                 float hz, bool& ok) {
    const float sx = x1x + hl * ex, sy = x1y + hl * ey, sz = x1z + hl * ez;   // x1 - xs
    const float rx = x1x - hl * ex, ry = x1y - hl * ey, rz = x1z - hl * ez;   // x1 - xr
    const float ss = sx * sx + sy * sy + sz * sz, rr = rx * rx + ry * ry + rz * rz;
    ok = (ss > 1e-12f) && (rr > 1e-12f);
    // approximate reciprocal square roots (relative error ~1e-7): the bound's error is a few
    // 1e-5 band units at most, far inside CULL_MARGIN
    const float is = rsqrt_approx(fmaxf(ss, 1e-12f)), ir = rsqrt_approx(fmaxf(rr, 1e-12f));
    const float gx = sx * is + rx * ir, gy = sy * is + ry * ir, gz = sz * is + rz * ir;
    const float lin = gx * (cx - x1x) + gy * (cy - x1y) + gz * (cz - x1z);
    return (ss * is + rr * ir - 2.0f * hl) + lin - (fabsf(gx) * hx + fabsf(gy) * hy + fabsf(gz) * hz);
}

__device__ __forceinline__ bool box_may_touch(float dx, float dy, float dz, float ex, float ey,
                                              float ez, float hl, float hx, float hy, float hz) {
    const float sx = dx + hl * ex, sy = dy + hl * ey, sz = dz + hl * ez;   // c - xs
    const float rx = dx - hl * ex, ry = dy - hl * ey, rz = dz - hl * ez;   // c - xr
    const float ss = sx * sx + sy * sy + sz * sz, rr = rx * rx + ry * ry + rz * rz;
    if (!(ss > 1e-12f) || !(rr > 1e-12f)) return true;
    const float is = rsqrt_approx(ss), ir = rsqrt_approx(rr);
    const float Rs = ss * is, Rr = rr * ir;
    const float gx = sx * is + rx * ir, gy = sy * is + ry * ir, gz = sz * is + rz * ir;
    const float lb = (Rs + Rr - 2.0f * hl) - (fabsf(gx) * hx + fabsf(gy) * hy + fabsf(gz) * hz);
    if (!(lb < 1.0f + CULL_MARGIN)) return false;   // NaN keeps the entry
    // second plane at the corner x1 = c - sign(grad R(c)) * half
    const float x1x = dx - copysignf(hx, gx), x1y = dy - copysignf(hy, gy), x1z = dz - copysignf(hz, gz);
    bool ok;
    const float lb1 = tangent_box_min(x1x, x1y, x1z, dx, dy, dz, ex, ey, ez, hl, hx, hy, hz, ok);
    return !(ok && lb1 >= 1.0f + CULL_MARGIN);
}

// Normalised detour v = R / U in [0, 1] (saturated) and the two inverse distances, from
// the pair-frame coordinates of a voxel centre: p = (x - o).e, q2 = |(x - o) x e|^2.
//   STABLE: R = q2 (A + B) / (A B) + E with A = R_xs + |p + hl|, B = R_xr + |p - hl| and
//           E = (|p + hl| - (p + hl)) + (|p - hl| + (p - hl)); every term is >= 0, so there
//           is no cancellation near the ray (R_xs - |ps| = q2 / (R_xs + |ps|)).
//   NAIVE:  R = R_xs + R_xr - 2 hl by subtraction.
// INNER: the caller guarantees |p| <= hl (the voxel lies between the planes through the two
// transducers normal to the pair axis); then E = 0 and the absolute values drop out.
// The caller passes ps = p + hl and pr = p - hl (the axial offsets from the emitter and the
// receiver) directly, so that they can be stepped along a run of voxels.
// RAW: return R / U unsaturated (the caller clamps), so that values just above 1 stay visible.
// GUARD: K0 has no single value at a transducer (its limit depends on the direction of
// approach); like the oracle, the guarded form gives 0 there. A voxel centre on a transducer
// lands ~1e-7 band units off it after FP32 rounding, where the plain form would evaluate a huge
// 1 / R_xs times a non-zero Phi; points within GUARD_R of a transducer are therefore taken as
// on it (is = ir = 0, so the entry is 0).
constexpr float GUARD_R2 = 1e-8f;   // (1e-4 band units)^2

template <int DT, bool GUARD, bool INNER = false, bool RAW = false>
__device__ __forceinline__ float detour_v(float ps, float pr, float q2, float hl, float& is, float& ir) {
    float ss = fmaf(ps, ps, q2), rr = fmaf(pr, pr, q2);
    bool at_tx = false;
    if (GUARD) {
        at_tx = (ss < GUARD_R2) || (rr < GUARD_R2);
        ss = fmaxf(ss, 1e-30f);
        rr = fmaxf(rr, 1e-30f);
    }
    is = rsqrt_approx(ss);
    ir = rsqrt_approx(rr);
    if (GUARD && at_tx) {
        is = 0.0f;
        ir = 0.0f;
        return 0.0f;
    }
    if (DT == FFT_DT_NAIVE) {
        const float v = fmaf(ss, is, fmaf(rr, ir, -2.0f * hl));
        return RAW ? v : __saturatef(v);
    } else if (INNER) {
        float A = fmaf(ss, is, ps), B = fmaf(rr, ir, -pr);
        float N = q2 * (A + B);
        const float v = N * rcp_approx(A * B);
        return RAW ? v : __saturatef(v);
    } else {
        float aps = fabsf(ps), apr = fabsf(pr);
        float A = fmaf(ss, is, aps), B = fmaf(rr, ir, apr);   // R_xs + |ps|, R_xr + |pr|
        float N = q2 * (A + B);
        float rP = rcp_approx(A * B);
        float E = (aps - ps) + (apr + pr);
        const float v = fmaf(N, rP, E);
        return RAW ? v : __saturatef(v);
    }
}

// In-support test dt < dt_max for voxel (ix, iy, iz) and a row given by its transducer
// positions, evaluated in FP64 with the cancellation-free detour (same arithmetic as the FP64
// oracle). Used only for the rare voxels whose FP32 detour lies within CUT_BAND of the cut-off
// of a band whose Phi does not vanish there, so that the in/out decision is taken in FP64.
static __device__ __forceinline__ bool in_support64(const RowRec64& r, double ox, double oy, double oz, double h, int ix,
                                          int iy, int iz, double U) {
    double x = ox + ix * h, y = oy + iy * h, z = oz + iz * h;
    double ex = r.xr[0] - r.xs[0], ey = r.xr[1] - r.xs[1], ez = r.xr[2] - r.xs[2];
    double L = sqrt(ex * ex + ey * ey + ez * ez);
    ex /= L; ey /= L; ez /= L;
    double dx = x - 0.5 * (r.xs[0] + r.xr[0]), dy = y - 0.5 * (r.xs[1] + r.xr[1]), dz = z - 0.5 * (r.xs[2] + r.xr[2]);
    double p = dx * ex + dy * ey + dz * ez;
    double c1 = dy * ez - dz * ey, c2 = dz * ex - dx * ez, c3 = dx * ey - dy * ex;
    double q2 = c1 * c1 + c2 * c2 + c3 * c3;
    double hl = 0.5 * L, ps = p + hl, pr = p - hl;
    double Rs = sqrt(ps * ps + q2), Rr = sqrt(pr * pr + q2);
    double A = Rs + fabs(ps), B = Rr + fabs(pr);
    double R = (q2 > 0.0 ? q2 * (A + B) / (A * B) : 0.0) + ((fabs(ps) - ps) + (fabs(pr) + pr));
    return R < U;
}

// Applies the FP64 decision to an FP32 normalised detour v near 1.
__device__ __forceinline__ float settle_cut(float v, bool in) {
    return in ? fminf(v, 0.99999994f) : 1.0f;
}

// One entry J[p, v] / C_p-free part times C_p, evaluated directly for voxel (ix, iy, iz) in FP32
// (pair frame from the row record; cancellation-free detour; FP64 cut decision for sharp bands
// when rec64 is given). Table lookup from global memory.
__device__ __forceinline__ float jentry_f32(const RowRec& r, const BandConst& c, const float2* __restrict__ tab,
                                            int n_tab, const RowRec64* rec64, int p, double ox, double oy,
                                            double oz, double h64, int ix, int iy, int iz, bool naive);

// Table lookup with linear interpolation, Phi(v) for the normalised detour v in [0, 1].
// Entry k of a band table holds (Phi_k - k dPhi_k, nm1 dPhi_k) with dPhi_k = Phi_{k+1} - Phi_k
// and nm1 = n_tab - 1, so that on [k, k + 1) / nm1 the interpolant is one FFMA in v:
//   Phi_k + (v nm1 - k) dPhi_k = (Phi_k - k dPhi_k) + v (nm1 dPhi_k).
// k = floor(v nm1) comes from a round-down add of MAGIC, whose bit pattern then addresses the
// table directly: tb is the shared-memory byte address of the band table minus (MAGIC bits << 3).
__device__ __forceinline__ float phi_lookup(float v, uint32_t tb, float nm1) {
    const float tt = __fmaf_rd(v, nm1, MAGIC);
    const float2 T = lds_f2(tb + (__float_as_uint(tt) << 3));
    return fmaf(v, T.y, T.x);
}

// Phi(v) from the band's sine series (Sec. II-C stored form): Phi = sum_{k=1..n} a_k sin(k x),
// x = theta v with theta = dw dt_max <= pi, and 0 for v <= 0 or v >= 1 (truncation).
// Block at shared address tb: theta, 3 pad floats, then a_1 .. a_{4 nq} (zeros past n).
// Clenshaw's recurrence b_k = a_k + 2 cos(x) b_{k+1} - b_{k+2} gives the sum as b_1 sin(x):
// two FP32 operations per term. sin(x) and 2 cos(x) come from Taylor polynomials in
// y = x - pi/2 in [-pi/2, pi/2] (sin x = cos y, cos x = -sin y; truncation below 1e-9), so
// that both stay accurate to a few FP32 ulps: the recurrence amplifies an error in cos(x) by
// up to ~n^2 near x = 0.
__device__ __forceinline__ float phi_trig(float v, uint32_t tb, int nq) {
    const float theta = lds_f1(tb);
    const float y = fmaf(theta, v, -1.57079632679489662f);
    const float y2 = y * y;
    // 2 cos x = -2 sin y = y (-2 + y^2 (2/3! - y^2 (2/5! - ...)))
    float c2 = fmaf(y2, -3.2118088e-10f, 5.0104217e-8f);      // -2/13!, 2/11!
    c2 = fmaf(c2, y2, -5.5114638e-6f);                         // -2/9!
    c2 = fmaf(c2, y2, 3.9682540e-4f);                          // 2/7!
    c2 = fmaf(c2, y2, -1.6666667e-2f);                         // -2/5!
    c2 = fmaf(c2, y2, 3.3333333e-1f);                          // 2/3!
    c2 = fmaf(c2, y2, -2.0f);
    c2 *= y;
    // sin x = cos y = 1 - y^2/2! + y^4/4! - ...
    float sx = fmaf(y2, 2.0876757e-9f, -2.7557319e-7f);        // 1/12!, -1/10!
    sx = fmaf(sx, y2, 2.4801587e-5f);                          // 1/8!
    sx = fmaf(sx, y2, -1.3888889e-3f);                         // -1/6!
    sx = fmaf(sx, y2, 4.1666667e-2f);                          // 1/4!
    sx = fmaf(sx, y2, -0.5f);
    sx = fmaf(sx, y2, 1.0f);
    float b1 = 0.0f, b2 = 0.0f;
    uint32_t pa = tb + 16u * (uint32_t)nq;   // group nq holds a_{4nq-3} .. a_{4nq}
#pragma unroll 2
    for (int q = nq; q > 0; --q, pa -= 16u) {
        const float4 a = lds_f4(pa);
        float b0 = fmaf(c2, b1, a.w - b2);
        b2 = fmaf(c2, b0, a.z - b1);
        b1 = fmaf(c2, b2, a.y - b0);
        b0 = fmaf(c2, b1, a.x - b2);
        // after the four steps: (b_k, b_{k+1}) = (b0, b1)
        b2 = b1;
        b1 = b0;
    }
    const float S = b1 * sx;
    return (v > 0.0f && v < 1.0f) ? S : 0.0f;
}

// phi_trig for N values of one band at once: the N recurrences run interleaved (independent
// chains for the scheduler) and share each shared-memory load of four coefficients.
template <int N>
__device__ __forceinline__ void phi_trig_n(const float* v, uint32_t tb, int nq, float* out) {
    const float theta = lds_f1(tb);
    float c2[N], sx[N], b1[N], b2[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float y = fmaf(theta, v[i], -1.57079632679489662f);
        const float y2 = y * y;
        float c = fmaf(y2, -3.2118088e-10f, 5.0104217e-8f);
        c = fmaf(c, y2, -5.5114638e-6f);
        c = fmaf(c, y2, 3.9682540e-4f);
        c = fmaf(c, y2, -1.6666667e-2f);
        c = fmaf(c, y2, 3.3333333e-1f);
        c = fmaf(c, y2, -2.0f);
        c2[i] = c * y;
        float t = fmaf(y2, 2.0876757e-9f, -2.7557319e-7f);
        t = fmaf(t, y2, 2.4801587e-5f);
        t = fmaf(t, y2, -1.3888889e-3f);
        t = fmaf(t, y2, 4.1666667e-2f);
        t = fmaf(t, y2, -0.5f);
        sx[i] = fmaf(t, y2, 1.0f);
        b1[i] = 0.0f;
        b2[i] = 0.0f;
    }
    uint32_t pa = tb + 16u * (uint32_t)nq;
    for (int q = nq; q > 0; --q, pa -= 16u) {
        const float4 a = lds_f4(pa);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float b0 = fmaf(c2[i], b1[i], a.w - b2[i]);
            float bb = fmaf(c2[i], b0, a.z - b1[i]);
            float ba = fmaf(c2[i], bb, a.y - b0);
            b0 = fmaf(c2[i], ba, a.x - bb);
            b2[i] = ba;
            b1[i] = b0;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = (v[i] > 0.0f && v[i] < 1.0f) ? b1[i] * sx[i] : 0.0f;
}

// The same from a band table in global memory (n_tab entries).
__device__ __forceinline__ float phi_lookup_global(float v, const float2* __restrict__ tab, int n_tab) {
    const float tt = __fmaf_rd(v, (float)(n_tab - 1), MAGIC);
    int k = (int)(__float_as_uint(tt) - 0x4B400000u);
    k = k < 0 ? 0 : (k > n_tab - 1 ? n_tab - 1 : k);
    const float2 T = tab[k];
    return fmaf(v, T.y, T.x);
}

}  // namespace fftgb

namespace fftgb {
__device__ __forceinline__ float jentry_f32(const RowRec& r, const BandConst& c, const float2* __restrict__ tab,
                                            int n_tab, const RowRec64* rec64, int p, double ox, double oy,
                                            double oz, double h64, int ix, int iy, int iz, bool naive) {
    const float dx = fmaf((float)ix, c.h, c.org[0]) - r.a.x;
    const float dy = fmaf((float)iy, c.h, c.org[1]) - r.a.y;
    const float dz = fmaf((float)iz, c.h, c.org[2]) - r.a.z;
    const float ex = r.b.x, ey = r.b.y, ez = r.b.z;
    const float pp = fmaf(dx, ex, fmaf(dy, ey, dz * ez));
    const float c1 = fmaf(dy, ez, -dz * ey), c2 = fmaf(dz, ex, -dx * ez), c3 = fmaf(dx, ey, -dy * ex);
    const float q2 = fmaf(c1, c1, fmaf(c2, c2, c3 * c3));
    float is, ir;
    float vv = naive ? detour_v<FFT_DT_NAIVE, true, false, true>(pp + r.a.w, pp - r.a.w, q2, r.a.w, is, ir)
                     : detour_v<FFT_DT_STABLE, true, false, true>(pp + r.a.w, pp - r.a.w, q2, r.a.w, is, ir);
    if (c.sharp && rec64 && fabsf(vv - 1.0f) < CUT_BAND)
        vv = settle_cut(__saturatef(vv), in_support64(rec64[p], ox, oy, oz, h64, ix, iy, iz, c.U));
    vv = __saturatef(vv);
    return phi_lookup_global(vv, tab, n_tab) * (is * ir) * r.b.w;
}
}  // namespace fftgb
