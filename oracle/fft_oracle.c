/*
 * FP64 CPU oracle for finite-frequency traveltime tomography (Korta Martiartu, Boehm and
 * Fichtner, "3D wave-equation-based finite-frequency tomography for ultrasound computed
 * tomography", arXiv:1908.03302).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously-correct definition
 * of what the CUDA library computes. Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Everything is double precision. Sums use Kahan compensation. OpenMP parallelises
 * over independent rows (J) or voxels (J^T); each output element is summed by one thread
 * in a fixed order, so results do not depend on the thread count.
 *
 * What each function follows:
 *   phi table      Sec. II-C, Eq. Kernel_freq: the spectrum-weighted frequency integral
 *                  Phi(dt) = int w^3 W(w) sin(w dt) dw / int w^2 W(w) dw, W = |f(w)|^2,
 *                  upper limits read as infinity; sampled at dt_k = k dt_max / (n-1).
 *   phi lookup     Sec. II-C: the operator is truncated at a maximum detour; Phi = 0 for
 *                  dt >= dt_max and for dt <= 0, linear interpolation in between.
 *   phi series     Sec. II-C: the alternative the paper stores, the coefficients and
 *                  arguments of the sine terms of Eq. Kernel_freq: both frequency integrals
 *                  by a rectangle rule on equally spaced nodes, Phi = sum_j a_j sin(w_j dt),
 *                  summed term by term in FP64, same truncation.
 *   detour         Sec. II-C: R = R_xs + R_xr - R_sr, dt = R / c0, evaluated in a form
 *                  with only non-negative terms (no cancellation near the ray).
 *   K0             Eq. Kernel_freq with A from Eq. Linearized_sensitivity:
 *                  K0 = -R_sr / (2 pi c0^3 R_xs R_xr) * Phi(dt).
 *   J, J^T         Eq. forward_compact / Eq. forward_ffttt: dT_p = sum_v K0(x_v) dV dc_v,
 *                  midpoint rule at voxel centres, dV = h^3; J^T is its transpose.
 *   CGLS           Sec. II-D, Eq. leastSquare_misfit with Gamma_n = I, Gamma_pr = I:
 *                  minimise 1/2 |J m - d|^2 + 1/2 lambda |m|^2 by conjugate gradients on
 *                  the damped normal equations (CGLS form), m0 = 0, fixed iterations.
 *   PSF            Sec. II-D, Eq. resolution_2: the Hessian H = J^T J applied to a
 *                  point-localised perturbation e_k, over a subset of rows.
 *   coverage       Sec. III-A: the absolute values of the operator's entries summed over
 *                  the rows, per voxel (the sensitivity coverage of an acquisition).
 *   J2, J2^T       Sec. II-B, Eq. forward_2D: the kernel integrated over z (midpoint rule on
 *                  the grid's layers) acting on a plane map dc(x, y).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ Kahan sums */
typedef struct { double s, c; } ksum;
static inline void kadd(ksum* k, double x) {
    double y = x - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* ------------------------------------------------------------------ spectrum */
/* Gaussian power spectrum, even extension to negative frequencies:
 * W(w) = exp(-(w-w0)^2/(2 s^2)) + exp(-(w+w0)^2/(2 s^2)), w0 = 2 pi fc, s = 2 pi sigma. */
static double w_gauss(double w, double w0, double s) {
    double a = (w - w0) / s, b = (w + w0) / s;
    return exp(-0.5 * a * a) + exp(-0.5 * b * b);
}

int oracle_n_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Phi table by quadrature (Eq. Kernel_freq).
 * kind 0: Gaussian W, composite Simpson over [0, w0 + 12 s] with n_quad (even) intervals.
 * kind 1: sampled W given at ascending nodes om[0..n_om-1]; trapezoid rule over the nodes.
 * out[k] = Phi(k dt_max / (n-1)), k = 0..n-1. Returns 0, or -1 on bad arguments.
 */
int oracle_phi_table(int kind, double fc, double fsig, const double* om, const double* W,
                     int n_om, int n_quad, int n, double dt_max, double* out) {
    if (n < 2 || !(dt_max > 0) || !out) return -1;
    if (kind == 0) {
        if (!(fc > 0) || !(fsig > 0) || n_quad < 2 || (n_quad & 1)) return -1;
        double w0 = 2 * ORC_PI * fc, s = 2 * ORC_PI * fsig;
        double wmax = w0 + 12 * s, dw = wmax / n_quad;
        ksum den = {0, 0};
        for (int q = 0; q <= n_quad; ++q) {
            double w = q * dw;
            double c = (q == 0 || q == n_quad) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
            kadd(&den, c * w * w * w_gauss(w, w0, s));
        }
        double D = den.s * dw / 3.0;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n; ++k) {
            double dt = k * dt_max / (n - 1);
            ksum num = {0, 0};
            for (int q = 0; q <= n_quad; ++q) {
                double w = q * dw;
                double c = (q == 0 || q == n_quad) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
                kadd(&num, c * w * w * w * w_gauss(w, w0, s) * sin(w * dt));
            }
            out[k] = (num.s * dw / 3.0) / D;
        }
        return 0;
    }
    if (kind == 1) {
        if (!om || !W || n_om < 2) return -1;
        ksum den = {0, 0};
        for (int q = 0; q + 1 < n_om; ++q) {
            double h = om[q + 1] - om[q];
            kadd(&den, 0.5 * h * (om[q] * om[q] * W[q] + om[q + 1] * om[q + 1] * W[q + 1]));
        }
#pragma omp parallel for schedule(static)
        for (int k = 0; k < n; ++k) {
            double dt = k * dt_max / (n - 1);
            ksum num = {0, 0};
            for (int q = 0; q + 1 < n_om; ++q) {
                double h = om[q + 1] - om[q];
                double a = om[q] * om[q] * om[q] * W[q] * sin(om[q] * dt);
                double b = om[q + 1] * om[q + 1] * om[q + 1] * W[q + 1] * sin(om[q + 1] * dt);
                kadd(&num, 0.5 * h * (a + b));
            }
            out[k] = num.s / den.s;
        }
        return 0;
    }
    return -1;
}

/*
 * Sine-series form of Phi (Sec. II-C, Eq. Kernel_freq), Gaussian spectrum.
 * Nodes w_j = j dw, j = 1..n; with the rectangle rule for both integrals
 *   Phi(dt) = sum_j a_j sin(w_j dt),   a_j = dw w_j^3 W(w_j) / int_0^inf w^2 W(w) dw,
 * the denominator by the composite Simpson rule of oracle_phi_table (n_quad intervals).
 * The rule is exact up to aliasing from the period T = 2 pi / dw of the series and the
 * truncation of the terms (the paper says a small number of terms suffices, not which):
 *   T = max(2 dt_max, dt_max + 6.5 / s)   (Phi decays like exp(-s^2 t^2 / 2): images of
 *                                          Phi shifted by T are negligible on [0, dt_max]),
 *   n = ceil((w0 + 5.5 s) / dw)           (W < 3e-7 beyond; series error < 2e-8 of max |Phi|),
 *                                          unless n_terms > 0 is given.
 * a must hold n values (at most 4096). Returns 0, or -1 on bad arguments.
 */
int oracle_trig_coefs(double fc, double fsig, double dt_max, int n_terms, int n_quad, double* a,
                      double* dw_out, int* n_out) {
    if (!(fc > 0) || !(fsig > 0) || !(dt_max > 0) || n_quad < 2 || (n_quad & 1) || !a) return -1;
    double w0 = 2 * ORC_PI * fc, s = 2 * ORC_PI * fsig;
    double T = 2.0 * dt_max;
    if (dt_max + 6.5 / s > T) T = dt_max + 6.5 / s;
    double dw = 2 * ORC_PI / T;
    int n = n_terms > 0 ? n_terms : (int)ceil((w0 + 5.5 * s) / dw);
    if (n < 1 || n > 4096) return -1;
    double wmax = w0 + 12 * s, hq = wmax / n_quad;
    ksum den = {0, 0};
    for (int q = 0; q <= n_quad; ++q) {
        double w = q * hq;
        double c = (q == 0 || q == n_quad) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
        kadd(&den, c * w * w * w_gauss(w, w0, s));
    }
    double D = den.s * hq / 3.0;
    for (int j = 1; j <= n; ++j) {
        double w = j * dw;
        a[j - 1] = dw * w * w * w * w_gauss(w, w0, s) / D;
    }
    if (dw_out) *dw_out = dw;
    if (n_out) *n_out = n;
    return 0;
}

/* The truncated series: 0 for dt <= 0 or dt >= dt_max, else sum_j a_j sin(j dw dt). */
double oracle_phi_trig(const double* a, int n, double dw, double dt_max, double dt) {
    if (!(dt > 0.0) || dt >= dt_max) return 0.0;
    ksum acc = {0, 0};
    for (int j = 1; j <= n; ++j) kadd(&acc, a[j - 1] * sin(j * dw * dt));
    return acc.s;
}

/* Truncated, linearly interpolated Phi (Sec. II-C truncation). */
double oracle_phi(const double* tab, int n, double dt_max, double dt) {
    if (!(dt > 0.0) || dt >= dt_max) return 0.0;
    double u = dt * (double)(n - 1) / dt_max;
    int i = (int)floor(u);
    if (i >= n - 1) return 0.0;
    double f = u - (double)i;
    return tab[i] + f * (tab[i + 1] - tab[i]);
}

/*
 * Detour R = R_xs + R_xr - R_sr for a point x and the pair (xs, xr), written with only
 * non-negative terms. With o the pair midpoint, e the unit axis, half-length hl = L/2,
 * p = (x - o).e and q2 = |(x - o) x e|^2:
 *   R_xs = sqrt((p+hl)^2 + q2), R_xr = sqrt((p-hl)^2 + q2),
 *   |p| <= hl:  R = q2/(R_xs+p+hl) + q2/(R_xr+hl-p)
 *   |p| >  hl:  R = 2(|p|-hl) + q2/(R_far+|p|+hl) + q2/(R_near+|p|-hl),
 *               R_far / R_near the distances to the transducer farther from / nearer to x.
 */
void oracle_detour(const double* xs, const double* xr, const double* x,
                   double* R, double* Rxs, double* Rxr, double* L_out) {
    double e[3] = {xr[0] - xs[0], xr[1] - xs[1], xr[2] - xs[2]};
    double L = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    e[0] /= L; e[1] /= L; e[2] /= L;
    double d[3] = {x[0] - 0.5 * (xs[0] + xr[0]), x[1] - 0.5 * (xs[1] + xr[1]),
                   x[2] - 0.5 * (xs[2] + xr[2])};
    double p = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    double c0 = d[1] * e[2] - d[2] * e[1];
    double c1 = d[2] * e[0] - d[0] * e[2];
    double c2 = d[0] * e[1] - d[1] * e[0];
    double q2 = c0 * c0 + c1 * c1 + c2 * c2;
    double hl = 0.5 * L;
    double rs = sqrt((p + hl) * (p + hl) + q2);
    double rr = sqrt((p - hl) * (p - hl) + q2);
    /* Terms are grouped so that swapping emitter and receiver (p -> -p, rs <-> rr) gives
     * bit-identical results: both cases below are symmetric under that swap. */
    double r;
    double ap = fabs(p);
    if (q2 == 0.0) {
        r = (ap <= hl) ? 0.0 : 2.0 * (ap - hl);
    } else if (ap <= hl) {
        r = q2 / (rs + (hl + p)) + q2 / (rr + (hl - p));
    } else {
        double far = (p > 0.0) ? rs : rr, near = (p > 0.0) ? rr : rs;
        double u = ap - hl, w = ap + hl;
        r = (2.0 * u + q2 / (far + w)) + q2 / (near + u);
    }
    *R = r; *Rxs = rs; *Rxr = rr;
    if (L_out) *L_out = L;
}

/* Detour by the textbook formula |x-xs| + |x-xr| - |xs-xr| (used only as a cross-check). */
double oracle_detour_naive(const double* xs, const double* xr, const double* x) {
    double a = sqrt((x[0] - xs[0]) * (x[0] - xs[0]) + (x[1] - xs[1]) * (x[1] - xs[1]) +
                    (x[2] - xs[2]) * (x[2] - xs[2]));
    double b = sqrt((x[0] - xr[0]) * (x[0] - xr[0]) + (x[1] - xr[1]) * (x[1] - xr[1]) +
                    (x[2] - xr[2]) * (x[2] - xr[2]));
    double L = sqrt((xs[0] - xr[0]) * (xs[0] - xr[0]) + (xs[1] - xr[1]) * (xs[1] - xr[1]) +
                    (xs[2] - xr[2]) * (xs[2] - xr[2]));
    return a + b - L;
}

/* Is x exactly on one of the transducers? Tested on the coordinates themselves: the distances
 * rebuilt in the pair frame round to ~1e-18 m instead of 0 there. */
static int on_transducer(const double* xs, const double* xr, const double* x) {
    return (x[0] == xs[0] && x[1] == xs[1] && x[2] == xs[2]) || (x[0] == xr[0] && x[1] == xr[1] && x[2] == xr[2]);
}

/* K0(x; xs, xr) of Eq. Kernel_freq (units s^2 / m^4). Zero at the transducers (its limit there
 * depends on the direction of approach; Phi(0) = 0 makes the limit along the ray zero). */
double oracle_k0(const double* xs, const double* xr, const double* x, double c0,
                 const double* tab, int n, double dt_max) {
    double R, rs, rr, L;
    if (on_transducer(xs, xr, x)) return 0.0;
    oracle_detour(xs, xr, x, &R, &rs, &rr, &L);
    if (rs == 0.0 || rr == 0.0) return 0.0;
    double phi = oracle_phi(tab, n, dt_max, R / c0);
    return -L / (2.0 * ORC_PI * c0 * c0 * c0 * (rs * rr)) * phi;
}

/* ------------------------------------------------------------------ operator */
typedef struct {
    const double* tx;        /* n_tx x 3 */
    const int32_t* rows;     /* M x 2 (s, r) */
    const int32_t* band;     /* M, nullable (all band 0) */
    const double* tables;    /* n_bands x n */
    const double* dt_max;    /* n_bands */
    int32_t n_tab;           /* samples per table */
    int32_t nx, ny, nz;
    double h;
    double org[3];
    double c0;
    const double* trig_dw;   /* n_bands, nullable: NULL = sampled tables; else tables hold the
                                n_tab sine-series coefficients of each band, node spacing dw */
} orc_geom;

static void vox_centre(const orc_geom* g, int64_t v, double* x) {
    int64_t i = v % g->nx, j = (v / g->nx) % g->ny, k = v / ((int64_t)g->nx * g->ny);
    x[0] = g->org[0] + (double)i * g->h;
    x[1] = g->org[1] + (double)j * g->h;
    x[2] = g->org[2] + (double)k * g->h;
}

/* Index box [lo, hi] (inclusive, clamped) enclosing the ellipsoid R <= c0 dt_max of row p,
 * widened by one voxel; voxels outside it have K0 = 0 exactly. Returns 0 if empty. */
static int row_box(const orc_geom* g, int64_t p, int64_t lo[3], int64_t hi[3]) {
    const double* xs = g->tx + 3 * (int64_t)g->rows[2 * p];
    const double* xr = g->tx + 3 * (int64_t)g->rows[2 * p + 1];
    int b = g->band ? g->band[p] : 0;
    double Rmax = g->c0 * g->dt_max[b];
    double e[3] = {xr[0] - xs[0], xr[1] - xs[1], xr[2] - xs[2]};
    double L = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    double a = 0.5 * (L + Rmax);
    double b2 = a * a - 0.25 * L * L;
    int n[3] = {g->nx, g->ny, g->nz};
    for (int ax = 0; ax < 3; ++ax) {
        double ek = (L > 0) ? e[ax] / L : 0.0;
        double ext = sqrt(a * a * ek * ek + b2 * (1.0 - ek * ek));
        double o = 0.5 * (xs[ax] + xr[ax]);
        double l = floor((o - ext - g->org[ax]) / g->h) - 1.0;
        double u = ceil((o + ext - g->org[ax]) / g->h) + 1.0;
        if (l < 0) l = 0;
        if (u > n[ax] - 1) u = n[ax] - 1;
        if (l > u) return 0;
        lo[ax] = (int64_t)l; hi[ax] = (int64_t)u;
    }
    return 1;
}

static inline double jentry(const orc_geom* g, int64_t p, const double* x) {
    const double* xs = g->tx + 3 * (int64_t)g->rows[2 * p];
    const double* xr = g->tx + 3 * (int64_t)g->rows[2 * p + 1];
    int b = g->band ? g->band[p] : 0;
    const double* tab = g->tables + (int64_t)b * g->n_tab;
    if (g->trig_dw) {   /* K0 with the sine-series Phi */
        double R, rs, rr, L;
        if (on_transducer(xs, xr, x)) return 0.0;
        oracle_detour(xs, xr, x, &R, &rs, &rr, &L);
        if (rs == 0.0 || rr == 0.0) return 0.0;
        double phi = oracle_phi_trig(tab, g->n_tab, g->trig_dw[b], g->dt_max[b], R / g->c0);
        return -L / (2.0 * ORC_PI * g->c0 * g->c0 * g->c0 * (rs * rr)) * phi * g->h * g->h * g->h;
    }
    return oracle_k0(xs, xr, x, g->c0, tab, g->n_tab, g->dt_max[b]) * g->h * g->h * g->h;
}

#define GEOM_ARGS const double *tx, const int32_t *rows, const int32_t *band, \
    const double *tables, const double *dt_max, int32_t n_tab, int32_t nx, int32_t ny, \
    int32_t nz, double h, const double *org, double c0, const double *trig_dw
#define GEOM_INIT orc_geom G = {tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, \
    {org[0], org[1], org[2]}, c0, trig_dw}; const orc_geom* g = &G

/* J entry for (row p, voxel v). */
double oracle_J_entry(GEOM_ARGS, int64_t p, int64_t v) {
    GEOM_INIT;
    double x[3];
    vox_centre(g, v, x);
    return jentry(g, p, x);
}

/* d[i] = sum_v J[row_idx[i], v] m[v] for i < n_sel (row_idx NULL: all M rows). */
void oracle_J(GEOM_ARGS, int64_t M, const int64_t* row_idx, int64_t n_sel,
              const double* m, double* d) {
    GEOM_INIT;
    int64_t n_out = row_idx ? n_sel : M;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t p = row_idx ? row_idx[i] : i;
        int64_t lo[3], hi[3];
        ksum acc = {0, 0};
        if (row_box(g, p, lo, hi)) {
            for (int64_t k = lo[2]; k <= hi[2]; ++k)
                for (int64_t j = lo[1]; j <= hi[1]; ++j)
                    for (int64_t ii = lo[0]; ii <= hi[0]; ++ii) {
                        int64_t v = (k * g->ny + j) * g->nx + ii;
                        double x[3];
                        vox_centre(g, v, x);
                        double jv = jentry(g, p, x);
                        if (jv != 0.0) kadd(&acc, jv * m[v]);
                    }
        }
        d[i] = acc.s;
    }
}

/* g[i] = sum_p J[p, vox_idx[i]] d[p] over all M rows (vox_idx NULL: all voxels). */
void oracle_JT(GEOM_ARGS, int64_t M, const double* d, const int64_t* vox_idx, int64_t n_sel,
               double* gout) {
    GEOM_INIT;
    int64_t V = (int64_t)nx * ny * nz;
    int64_t n_out = vox_idx ? n_sel : V;
    int64_t* box = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(M > 0 ? M : 1));
    char* ok = (char*)malloc((size_t)(M > 0 ? M : 1));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < M; ++p) ok[p] = (char)row_box(g, p, box + 6 * p, box + 6 * p + 3);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t v = vox_idx ? vox_idx[i] : i;
        int64_t vi = v % nx, vj = (v / nx) % ny, vk = v / ((int64_t)nx * ny);
        double x[3];
        vox_centre(g, v, x);
        ksum acc = {0, 0};
        for (int64_t p = 0; p < M; ++p) {
            const int64_t* b = box + 6 * p;
            if (!ok[p] || d[p] == 0.0 || vi < b[0] || vi > b[3] || vj < b[1] || vj > b[4] ||
                vk < b[2] || vk > b[5])
                continue;
            double jv = jentry(g, p, x);
            if (jv != 0.0) kadd(&acc, jv * d[p]);
        }
        gout[i] = acc.s;
    }
    free(box);
    free(ok);
}

/* 2-D approximation (Sec. II-B, Eq. forward_2D): the kernel integrated over z by the midpoint
 * rule on the grid's nz layers, times a plane map m2[j * nx + i]:
 *   J2[p, (i, j)] = sum_k K0(x_i, y_j, z_k) h^3  (= h^2 * the z integral with spacing h). */
void oracle_J2d(GEOM_ARGS, int64_t M, const int64_t* row_idx, int64_t n_sel, const double* m2, double* d) {
    GEOM_INIT;
    int64_t n_out = row_idx ? n_sel : M;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t p = row_idx ? row_idx[i] : i;
        int64_t lo[3], hi[3];
        ksum acc = {0, 0};
        if (row_box(g, p, lo, hi)) {
            for (int64_t k = lo[2]; k <= hi[2]; ++k)
                for (int64_t j = lo[1]; j <= hi[1]; ++j)
                    for (int64_t ii = lo[0]; ii <= hi[0]; ++ii) {
                        double x[3];
                        vox_centre(g, (k * g->ny + j) * g->nx + ii, x);
                        double jv = jentry(g, p, x);
                        if (jv != 0.0) kadd(&acc, jv * m2[j * g->nx + ii]);
                    }
        }
        d[i] = acc.s;
    }
}

/* g2[(i, j)] = sum_p J2[p, (i, j)] d[p] for the pixels in pix_idx (NULL: all nx * ny). */
void oracle_JT2d(GEOM_ARGS, int64_t M, const double* d, const int64_t* pix_idx, int64_t n_sel, double* g2) {
    GEOM_INIT;
    int64_t n2 = (int64_t)nx * ny;
    int64_t n_out = pix_idx ? n_sel : n2;
    int64_t* box = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(M > 0 ? M : 1));
    char* ok = (char*)malloc((size_t)(M > 0 ? M : 1));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < M; ++p) ok[p] = (char)row_box(g, p, box + 6 * p, box + 6 * p + 3);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t u = pix_idx ? pix_idx[i] : i;
        int64_t vi = u % nx, vj = u / nx;
        ksum acc = {0, 0};
        for (int64_t p = 0; p < M; ++p) {
            const int64_t* b = box + 6 * p;
            if (!ok[p] || d[p] == 0.0 || vi < b[0] || vi > b[3] || vj < b[1] || vj > b[4]) continue;
            for (int64_t k = b[2]; k <= b[5]; ++k) {
                double x[3];
                vox_centre(g, (k * ny + vj) * nx + vi, x);
                double jv = jentry(g, p, x);
                if (jv != 0.0) kadd(&acc, jv * d[p]);
            }
        }
        g2[i] = acc.s;
    }
    free(box);
    free(ok);
}

/* The z integral of K0 at plane point (x, y) by the midpoint rule: nz nodes z0 + (k + 1/2) hz
 * (s^2 / m^3); used to pin the 2-D rule's convergence. */
double oracle_k2_midpoint(const double* xs, const double* xr, double x, double y, double z0, double hz, int nz,
                          double c0, const double* tab, int n, double dt_max) {
    ksum acc = {0, 0};
    for (int k = 0; k < nz; ++k) {
        double pt[3] = {x, y, z0 + (k + 0.5) * hz};
        kadd(&acc, oracle_k0(xs, xr, pt, c0, tab, n, dt_max) * hz);
    }
    return acc.s;
}

/* Sensitivity coverage (Sec. III-A): cov[i] = sum_p |J[p, vox_idx[i]] w[p]| over all M rows
 * (w NULL: all ones; vox_idx NULL: all voxels). */
void oracle_coverage(GEOM_ARGS, int64_t M, const double* w, const int64_t* vox_idx, int64_t n_sel,
                     double* cov) {
    GEOM_INIT;
    int64_t V = (int64_t)nx * ny * nz;
    int64_t n_out = vox_idx ? n_sel : V;
    int64_t* box = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(M > 0 ? M : 1));
    char* ok = (char*)malloc((size_t)(M > 0 ? M : 1));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < M; ++p) ok[p] = (char)row_box(g, p, box + 6 * p, box + 6 * p + 3);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t v = vox_idx ? vox_idx[i] : i;
        int64_t vi = v % nx, vj = (v / nx) % ny, vk = v / ((int64_t)nx * ny);
        double x[3];
        vox_centre(g, v, x);
        ksum acc = {0, 0};
        for (int64_t p = 0; p < M; ++p) {
            const int64_t* b = box + 6 * p;
            if (!ok[p] || vi < b[0] || vi > b[3] || vj < b[1] || vj > b[4] || vk < b[2] || vk > b[5]) continue;
            double wp = w ? w[p] : 1.0;
            if (wp == 0.0) continue;
            kadd(&acc, fabs(jentry(g, p, x) * wp));
        }
        cov[i] = acc.s;
    }
    free(box);
    free(ok);
}

/* Number of (row, voxel) pairs with 0 < dt < dt_max over the rows in row_idx (NULL: all),
 * i.e. the in-support evaluations of one J (or J^T) application. */
int64_t oracle_count_support(GEOM_ARGS, int64_t M, const int64_t* row_idx, int64_t n_sel) {
    GEOM_INIT;
    int64_t n_out = row_idx ? n_sel : M, total = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total)
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t p = row_idx ? row_idx[i] : i;
        int64_t lo[3], hi[3];
        if (!row_box(g, p, lo, hi)) continue;
        const double* xs = g->tx + 3 * (int64_t)g->rows[2 * p];
        const double* xr = g->tx + 3 * (int64_t)g->rows[2 * p + 1];
        int b = g->band ? g->band[p] : 0;
        for (int64_t k = lo[2]; k <= hi[2]; ++k)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t ii = lo[0]; ii <= hi[0]; ++ii) {
                    double x[3], R, rs, rr, L;
                    vox_centre(g, (k * g->ny + j) * g->nx + ii, x);
                    oracle_detour(xs, xr, x, &R, &rs, &rr, &L);
                    if (R / g->c0 < g->dt_max[b]) total += 1;
                }
    }
    return total;
}

/* Squared Frobenius norm of J (over all M rows and all voxels). */
double oracle_frob2(GEOM_ARGS, int64_t M) {
    GEOM_INIT;
    double total = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total)
    for (int64_t p = 0; p < M; ++p) {
        int64_t lo[3], hi[3];
        ksum acc = {0, 0};
        if (row_box(g, p, lo, hi)) {
            for (int64_t k = lo[2]; k <= hi[2]; ++k)
                for (int64_t j = lo[1]; j <= hi[1]; ++j)
                    for (int64_t ii = lo[0]; ii <= hi[0]; ++ii) {
                        double x[3];
                        vox_centre(g, (k * g->ny + j) * g->nx + ii, x);
                        double jv = jentry(g, p, x);
                        kadd(&acc, jv * jv);
                    }
        }
        total += acc.s;
    }
    return total;
}

static double dot(const double* a, const double* b, int64_t n) {
    ksum s = {0, 0};
    for (int64_t i = 0; i < n; ++i) kadd(&s, a[i] * b[i]);
    return s.s;
}

/*
 * Damped CGLS (Sec. II-D): minimise 1/2 |J m - d|^2 + 1/2 lambda |m|^2, m0 given in m
 * (pass zeros for m0 = 0), n_iter iterations, no early stop.
 *   r = d - J m; s = J^T r - lambda m; p = s; gamma = |s|^2
 *   loop: q = J p; delta = |q|^2 + lambda |p|^2; alpha = gamma / delta;
 *         m += alpha p; r -= alpha q; s = J^T r - lambda m;
 *         gamma' = |s|^2; beta = gamma' / gamma; p = s + beta p
 * hist (nullable, n_iter + 1 values) receives gamma before each iteration and at the end.
 * gamma = 0 means the gradient of the damped misfit vanishes at m: m is already its minimiser
 * (the misfit is a convex quadratic), so the remaining iterations leave m unchanged and record
 * gamma = 0. Returns 0, or -4 if delta <= 0 with a non-zero gradient or gamma is not finite.
 */
int oracle_cgls(GEOM_ARGS, int64_t M, const double* dobs, double lambda, int32_t n_iter,
                double* m, double* hist) {
    int64_t V = (int64_t)nx * ny * nz;
    double* r = (double*)malloc(sizeof(double) * (size_t)M);
    double* q = (double*)malloc(sizeof(double) * (size_t)M);
    double* s = (double*)malloc(sizeof(double) * (size_t)V);
    double* p = (double*)malloc(sizeof(double) * (size_t)V);
    int status = 0;
    oracle_J(tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, org, c0, trig_dw, M, NULL, 0, m, r);
    for (int64_t i = 0; i < M; ++i) r[i] = dobs[i] - r[i];
    oracle_JT(tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, org, c0, trig_dw, M, r, NULL, 0, s);
    for (int64_t v = 0; v < V; ++v) { s[v] -= lambda * m[v]; p[v] = s[v]; }
    double gamma = dot(s, s, V);
    if (hist) hist[0] = gamma;
    for (int32_t it = 0; it < n_iter; ++it) {
        if (!isfinite(gamma)) { status = -4; break; }
        if (gamma == 0.0) {   /* converged: m minimises the damped misfit */
            if (hist)
                for (int32_t k = it + 1; k <= n_iter; ++k) hist[k] = 0.0;
            break;
        }
        oracle_J(tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, org, c0, trig_dw, M, NULL, 0, p, q);
        double delta = dot(q, q, M) + lambda * dot(p, p, V);
        if (!(delta > 0.0)) { status = -4; break; }
        double alpha = gamma / delta;
        for (int64_t v = 0; v < V; ++v) m[v] += alpha * p[v];
        for (int64_t i = 0; i < M; ++i) r[i] -= alpha * q[i];
        oracle_JT(tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, org, c0, trig_dw, M, r, NULL, 0, s);
        for (int64_t v = 0; v < V; ++v) s[v] -= lambda * m[v];
        double gnew = dot(s, s, V);
        double beta = gnew / gamma;
        for (int64_t v = 0; v < V; ++v) p[v] = s[v] + beta * p[v];
        gamma = gnew;
        if (hist) hist[it + 1] = gamma;
    }
    free(r); free(q); free(s); free(p);
    return status;
}

/*
 * Hessian point-spread functions (Eq. resolution_2): for each spike voxel k and each row
 * subset S, psf[v] = sum_{p in S} J[p, v] J[p, k] (a unit 1 m/s spike). Subset rows are
 * given as CSR (sub_off[n_sub+1], sub_idx). Output out[(s * n_spike + k) * n_vox_sel + i]
 * for the selected voxels vox_idx[i] (NULL: all voxels, n_vox_sel = V).
 */
void oracle_psf(GEOM_ARGS, int64_t M, const int64_t* spikes, int32_t n_spike,
                const int32_t* sub_off, int32_t n_sub, const int32_t* sub_idx,
                const int64_t* vox_idx, int64_t n_vox_sel, double* out) {
    GEOM_INIT;
    int64_t V = (int64_t)nx * ny * nz;
    int64_t nv = vox_idx ? n_vox_sel : V;
    double* dcol = (double*)calloc((size_t)(M > 0 ? M : 1), sizeof(double));
    for (int32_t sb = 0; sb < n_sub; ++sb) {
        for (int32_t k = 0; k < n_spike; ++k) {
            double xk[3];
            vox_centre(g, spikes[k], xk);
            memset(dcol, 0, sizeof(double) * (size_t)M);
            for (int32_t t = sub_off[sb]; t < sub_off[sb + 1]; ++t) {
                int64_t p = sub_idx[t];
                dcol[p] = jentry(g, p, xk);
            }
            double* o = out + ((int64_t)sb * n_spike + k) * nv;
            oracle_JT(tx, rows, band, tables, dt_max, n_tab, nx, ny, nz, h, org, c0, trig_dw, M, dcol,
                      vox_idx, nv, o);
        }
    }
    free(dcol);
}
