/*
 * fft_gb300.h - C ABI of the GB300 (sm_103a) finite-frequency traveltime tomography library.
 *
 * The library applies the linearised cross-correlation traveltime operator of
 * Korta Martiartu, Boehm and Fichtner, "3D wave-equation-based finite-frequency tomography
 * for ultrasound computed tomography" (arXiv:1908.03302):
 *
 *   dT_p = sum_v J[p, v] dc_v,   J[p, v] = K0(x_v; x_s(p), x_r(p)) * h^3           (Eq. forward_compact)
 *   K0(x) = A(x) * Phi(dt),      A = -R_sr / (2 pi c0^3 R_xs R_xr)                 (Eq. Linearized_sensitivity)
 *   Phi(dt) = int w^3 W(w) sin(w dt) dw / int w^2 W(w) dw, W = |f(w)|^2             (Eq. Kernel_freq)
 *   dt = (R_xs + R_xr - R_sr) / c0, Phi = 0 for dt >= dt_max (truncation)          (Sec. II-C)
 *
 * and its adjoint, without ever storing J (entries are rebuilt on the fly in every call,
 * Sec. II-C), a damped least-squares CG solve (Sec. II-D, Eq. leastSquare_misfit) and
 * Hessian point-spread functions H e_k = J^T J e_k (Sec. II-D, Eq. resolution_2).
 *
 * Conventions shared by every call
 *   - Units are SI at the boundary: metres, seconds, m/s.
 *   - Rows (measurements) are emitter/receiver pairs in the caller's order; a row may carry a
 *     frequency band (its own Phi table). Voxels are the centres of a regular grid,
 *     v = (k * ny + j) * nx + i, x fastest; voxel (i, j, k) sits at origin + (i, j, k) * h.
 *   - Vectors m (length V = nx*ny*nz, m/s) and d (length M, s) are float32 device arrays
 *     owned by the caller. Handles own everything else (tables, pair records, cull lists,
 *     scratch), allocated at creation on the current device.
 *   - All apply/solve calls are asynchronous on the caller's CUDA stream (cudaStream_t passed
 *     as void*, NULL = legacy default stream) unless stated otherwise. A handle may be used
 *     by one stream at a time: its scratch buffers are shared by its calls.
 *   - Every call returns an fft_status; on failure fft_last_error() gives a message
 *     (thread-local). No C++ exception crosses this boundary.
 */
#ifndef FFT_GB300_H
#define FFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fft_status;
#define FFT_OK 0
#define FFT_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, bad mode) */
#define FFT_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define FFT_ERR_OOM (-3)       /* device allocation failed */
#define FFT_ERR_BREAKDOWN (-4) /* CG breakdown: a curvature <= 0 or a non-finite scalar */
#define FFT_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define FFT_ERR_STATE (-6)     /* handle in the wrong state (e.g. used on another device) */

/* Detour-time arithmetic inside the J / J^T kernels (chosen per geometry). */
#define FFT_DT_STABLE 0 /* FP32, cancellation-free form in the pair frame (default) */
#define FFT_DT_NAIVE 1  /* FP32, R_xs + R_xr - L by plain subtraction */
#define FFT_DT_FP64 2   /* detour in FP64, rest in FP32 (slow; precision studies) */

/* Source power spectrum W(w) = |f(w)|^2 (Eq. Kernel_freq).
 *   kind 0: Gaussian in frequency, W = exp(-(w-w0)^2/(2 s^2)) + exp(-(w+w0)^2/(2 s^2)),
 *           w0 = 2 pi f_center_hz, s = 2 pi f_sigma_hz (even extension to w < 0).
 *   kind 1: sampled, W(omega[j]) = weight[j] at ascending angular frequencies (host arrays,
 *           n_omega >= 2, read during the call only). */
typedef struct {
    int32_t kind;
    double f_center_hz;
    double f_sigma_hz;
    const double* omega;
    const double* weight;
    int32_t n_omega;
} fft_spectrum;

/* Voxel grid: nx, ny, nz >= 1; h > 0 the spacing; origin the centre of voxel (0, 0, 0). */
typedef struct {
    int32_t nx, ny, nz;
    double h;
    double origin[3];
} fft_grid;

typedef struct fft_table_s* fft_table; /* opaque: one Phi representation (sampled table or sine series) */
typedef struct fft_geom_s* fft_geom;   /* opaque: rows + grid + tables + cull lists */

/*
 * fft_table_build - sample Phi(dt_k), dt_k = k dt_max / (n_samples - 1), k = 0..n-1,
 * by FP64 quadrature on the device (Eq. Kernel_freq with upper limits read as infinity;
 * the sampled table is what Sec. II-C stores in place of F).
 *   spec       spectrum (host struct; sampled arrays are host memory).
 *   n_samples  2 .. 65536 (4096 in the reference workloads).
 *   dt_max     cut-off detour time in s (> 0); Phi is 0 at and beyond it.
 *   host_out   nullable; if given, receives the n_samples FP64 values (the call then
 *              synchronises with the device).
 *   out        receives the new handle; release with fft_table_destroy.
 * Quadrature: kind 0 composite Simpson over [0, w0 + 12 s] with 40000 intervals; kind 1
 * trapezoid rule over the given nodes. Synchronous apart from the optional copy above.
 */
fft_status fft_table_build(const fft_spectrum* spec, int32_t n_samples, double dt_max,
                           double* host_out, fft_table* out);
void fft_table_destroy(fft_table t);

/*
 * fft_trig_build - Phi as a short sine series, the form Sec. II-C keeps (amplitudes and
 * frequencies of the sine terms of Eq. Kernel_freq) in place of a sampled table:
 *   Phi(dt) = sum_{j=1..n} a_j sin(j dw dt),  0 for dt <= 0 or dt >= dt_max,
 *   a_j = dw w_j^3 W(w_j) / int_0^inf w^2 W(w) dw,  w_j = j dw,
 * i.e. both integrals by the rectangle rule on equally spaced nodes (the denominator in
 * closed form for the Gaussian W). Node spacing dw = 2 pi / T with the period
 * T = max(2 dt_max, dt_max + 6.5 / s): shifted images of Phi (which decays like
 * exp(-s^2 t^2 / 2)) are then negligible on [0, dt_max], and x = dw dt stays in [0, pi].
 *   spec         Gaussian spectrum only (kind 0); kind 1 gives FFT_ERR_ARG.
 *   dt_max       cut-off detour time in s (> 0).
 *   n_terms      0: automatic, n = ceil((w0 + 5.5 s) / dw) (W < 3e-7 beyond, series within 2e-8
 *                of max |Phi|; 18..20 terms for the reference workloads); else 1 .. 256 terms.
 *   coef_out     nullable, host: receives the n FP64 coefficients a_1 .. a_n.
 *   dw_out       nullable, host: receives dw (rad/s).
 *   n_terms_out  nullable, host: receives n.
 *   out          receives the handle; release with fft_table_destroy.
 * Geometries built from series handles evaluate Phi on the fly by the Clenshaw recurrence
 * (one sine and one cosine per evaluation, two FP32 operations per term) instead of the
 * table lookup. Synchronous; host-only arithmetic.
 */
fft_status fft_trig_build(const fft_spectrum* spec, double dt_max, int32_t n_terms, double* coef_out,
                          double* dw_out, int32_t* n_terms_out, fft_table* out);

/*
 * fft_geom_create - set up the operator J for one acquisition (Eq. forward_compact):
 *   tx_xyz       host, n_tx x 3 transducer positions (m).
 *   rows         host, n_rows x 2 (s, r) transducer indices, s != r. Row order is the
 *                order of d.
 *   band_of_row  host, nullable (all rows use table 0), else n_rows table indices.
 *   grid         voxel grid (host struct).
 *   c0           background sound speed (m/s) > 0.
 *   tables       host array of n_tables handles (1..8). The kernels hold every table in shared
 *                memory: n_tables x n_samples x 8 bytes + 16 KB must fit in the device's per-CTA
 *                shared memory (227 KB on sm_103a: up to 6 tables of 4096 samples, 8 of 2048),
 *                else FFT_ERR_ARG.
 *   dt_mode      FFT_DT_STABLE / FFT_DT_NAIVE / FFT_DT_FP64.
 * Builds per-row records and the culled (tile, row) lists on the device: a (16x16x8 voxel
 * tile, row) entry is kept unless a lower bound of the detour over the tile (tangent plane
 * of the convex R at the tile centre) proves dt >= dt_max everywhere in it. Synchronous.
 * Fails with FFT_ERR_ARG for empty inputs, out-of-range indices or s == r.
 */
fft_status fft_geom_create(const double* tx_xyz, int32_t n_tx, const int32_t* rows,
                           int64_t n_rows, const int32_t* band_of_row, const fft_grid* grid,
                           double c0, const fft_table* tables, int32_t n_tables,
                           int32_t dt_mode, fft_geom* out);
/* (fft_geom_create, continued) tables must all be sampled tables (fft_table_build) or all sine
 * series (fft_trig_build); a series geometry needs dt_mode FFT_DT_STABLE and supports J, J^T,
 * the Frobenius norm and CG; fft_psf_batch and fft_psf_noalloc reject it (FFT_ERR_ARG). */
void fft_geom_destroy(fft_geom g);

/* Sizes and counters of a geometry (host struct filled synchronously). */
typedef struct {
    int64_t n_rows;          /* M */
    int64_t n_vox;           /* V */
    int64_t n_entries;       /* kept (tile, row) entries */
    int64_t n_items;         /* work items of one apply */
    int64_t support_evals;   /* (row, voxel) pairs with 0 <= dt < dt_max: in-support evaluations
                                of one J or J^T (counted on the device at creation) */
    int64_t scratch_bytes;   /* device bytes owned by the handle */
    int32_t dt_mode;
    int64_t evaluated_evals; /* (row, voxel) evaluations one apply performs after culling */
    int32_t phi_terms;       /* 0: sampled tables; else the largest sine-series length */
    double psf_tc_mma_flops; /* tensor-core MMA flops of the last fft_psf_batch call in mode 1:
                                2 x 128 x 96 x N per chunk of generated J tile, N the MMA width */
    double psf_tc_entries;   /* J entries that call generated: 128 voxels x 96 rows per chunk,
                                the stand-in rows of partial chunks included */
} fft_geom_info_t;
fft_status fft_geom_info(fft_geom g, fft_geom_info_t* info);

/* Result of fft_geom_autotune. */
typedef struct {
    int32_t items_per_cta; /* chosen work-item granularity (items per persistent CTA) */
    int32_t ctas_per_sm;   /* chosen persistent CTAs per SM of the J / J^T kernels */
    double ms_J, ms_JT;    /* their measured times with the chosen decomposition */
    int32_t n_tried;       /* candidates timed */
} fft_tune_info_t;

/*
 * fft_geom_autotune - pick the work decomposition of J and J^T for this geometry by timing
 * them on the device: a tile's candidate rows are cut into work items sized for 4, 8, 16, 32,
 * 64 or 128 items per persistent CTA (at least 64 rows each), with the most CTAs per SM that
 * fit or one fewer. The sizes are swept at the occupancy limit (stopping after two in a row
 * more than 2 % slower than the best), then the best size and its two neighbours with one CTA
 * per SM fewer: 2 to 9 candidates. Each runs J^T and J once timed (CUDA events on `stream`),
 * after one untimed pass unless the previous candidate's pair took over 20 ms, and the
 * fastest is kept. Results do not depend on the choice beyond rounding of the split J^T sums.
 * For geometries with a band whose Phi does not vanish at its cut-off, J and J^T run in one
 * CTA of up to 20 warps per SM whatever the candidate; the CTA count then only sets the item
 * granularity. Synchronous; allocates test vectors for the duration of the call; invalidates
 * a captured CG loop (the next fft_cg_solve captures again). info may be NULL.
 */
fft_status fft_geom_autotune(fft_geom g, void* stream, fft_tune_info_t* info);

/*
 * fft_J_apply - d = J m (Eq. forward_compact; m in m/s, d in s).
 *   m_dev  device float32[V]; d_dev device float32[M] (written entirely). No aliasing.
 * Each row's value is a fixed-order sum (deterministic, bit-reproducible run to run).
 */
fft_status fft_J_apply(fft_geom g, const float* m_dev, float* d_dev, void* stream);

/*
 * fft_JT_apply - g = J^T d (the adjoint used by the normal equations, Eq. leastSquare_misfit).
 *   d_dev device float32[M]; g_dev device float32[V] (written entirely). Gather per voxel,
 *   no atomics; deterministic.
 */
fft_status fft_JT_apply(fft_geom g, const float* d_dev, float* g_dev, void* stream);

/*
 * fft_J_apply_batch / fft_JT_apply_batch - J or J^T applied to n vectors at once (the
 * operator of Eq. forward_compact and its adjoint, for block methods such as the low-rank
 * eigensolver): every evaluated entry J[p, v] is used for four columns, so a group of four
 * costs little more than one application.
 *   m_dev  device float32, n columns of length V (column c at m_dev + c * V);
 *   d_dev  device float32, n columns of length M (column c at d_dev + c * M);
 *   g_dev  device float32, n columns of length V.
 * Columns are processed in groups of four; a remainder (and every column of geometries with
 * a non-stable detour mode) goes through the single-vector kernels. Each column matches the
 * single-vector call to rounding (same entries, same summation order). The first call
 * allocates the handle's four-column scratch (E * 32 + slots * 4 * 2048 floats).
 */
fft_status fft_J_apply_batch(fft_geom g, const float* m_dev, int32_t n, float* d_dev, void* stream);
fft_status fft_JT_apply_batch(fft_geom g, const float* d_dev, int32_t n, float* g_dev, void* stream);

/*
 * fft_coverage - sensitivity coverage cov_v = sum_p |J[p, v] w_p|: the absolute values of the
 * operator's entries summed over the rows for every voxel (Sec. III-A, the coverage map of
 * the experiment; with w = 1 it is J^T of |J| applied to ones).
 *   w_dev    device float32[M] row weights (e.g. a 0/1 mask of a row subset), or NULL for 1.
 *   cov_dev  device float32[V] (written entirely). Same gather as fft_JT_apply: no atomics,
 *            deterministic.
 */
fft_status fft_coverage(fft_geom g, const float* w_dev, float* cov_dev, void* stream);

/*
 * 2-D approximation (Sec. II-B, Eq. forward_2D): transducers in one plane, a model dc(x, y)
 * that varies slowly in z over the kernels' extent; the kernel is integrated over z in
 * [z0, z1] and the model lives on the plane. The geometry's grid supplies both: its nz layers
 * are the z-quadrature nodes (midpoint rule, spacing h, the same rule as the volume
 * integral), so J2[p, (i, j)] = sum_k J[p, (i, j, k)]. Choose the layers to cover the
 * kernels' main contribution (the truncated support of the longest pair reaches
 * |z| = sqrt(((L + c0 dt_max)/2)^2 - (L/2)^2)).
 *   fft_J2d_apply   m2_dev device float32[nx * ny] (plane map, x fastest) -> d_dev float32[M].
 *   fft_JT2d_apply  d_dev float32[M] -> g2_dev float32[nx * ny] (each pixel's sum over the
 *                   layers in a fixed order; deterministic).
 * Both use a volume scratch (V floats) owned by the geometry, allocated on first use; calls
 * on one geometry must not overlap (as for all its calls).
 */
fft_status fft_J2d_apply(fft_geom g, const float* m2_dev, float* d_dev, void* stream);
fft_status fft_JT2d_apply(fft_geom g, const float* d_dev, float* g2_dev, void* stream);

/*
 * fft_hessian_lowrank - the k dominant eigenpairs of the prior-preconditioned misfit Hessian
 * H = J^T J / sigma^2 (Sec. II-D, Eq. low_rank, with Gamma_pr = I and Gamma_n^{-1} =
 * I / sigma^2), by randomized subspace iteration (Halko, Martinsson and Tropp, SIAM Review 53,
 * 2011, Algorithms 4.4 and 5.3):
 *   Y = H Omega; n_power times { Q = orth(Y); Y = H Q }; Q = orth(Y);
 *   T = Q^T H Q = U diag(l) U^T; V_k = Q U_k for the k largest l.
 *   omega_dev  device float32, ell columns of length V (column j at omega_dev + j * V): the
 *              starting block, drawn by the caller (e.g. standard normal); read only.
 *   ell, k     1 <= k <= ell <= 256 (ell - k is the oversampling).
 *   n_power    0 .. 64 power iterations.
 *   sigma      noise standard deviation in s (> 0; 1 gives the eigenpairs of J^T J).
 *   vecs_dev   device float32, k columns of length V: orthonormal eigenvectors, largest first.
 *   eigvals    host double[k]: the eigenvalues, descending.
 * H is applied with the batch J and J^T kernels, four columns at a time ((n_power + 2) ell
 * columns in all); orth is three SVQB passes (Gram matrix in FP64, its eigendecomposition on
 * the host; directions below 1e-12 of the largest Gram eigenvalue are dropped, so a block
 * wider than the rank of H is fine and yields zero Ritz values); the ell x ell eigenproblem is
 * solved on the host (cyclic Jacobi, FP64). Synchronous. Allocates two V x ell float32 blocks
 * and small buffers per call. FFT_ERR_BREAKDOWN if a block is zero or not finite.
 */
fft_status fft_hessian_lowrank(fft_geom g, const float* omega_dev, int32_t ell, int32_t k, int32_t n_power,
                               double sigma, float* vecs_dev, double* eigvals, void* stream);

/*
 * fft_lowrank_diag - diagonals of the low-rank posterior covariance and resolution matrix
 * (Eqs. posterior_app and resolution_app with Gamma_pr = I) from k eigenpairs of H:
 *   res_v = sum_i d_i V[v, i]^2,  post_v = (1 - res_v) / alpha,  d_i = l_i / (l_i + alpha).
 *   vecs_dev  device float32, k columns of length V; eigvals host double[k]; alpha > 0 the
 *             damping of Eq. leastSquare_misfit.
 *   post_dev, res_dev  device float32[V] outputs; either may be NULL. Synchronous.
 */
fft_status fft_lowrank_diag(fft_geom g, const float* vecs_dev, const double* eigvals, int32_t k, double alpha,
                            float* post_dev, float* res_dev, void* stream);

/*
 * fft_frob2 - |J|_F^2 = sum over rows and voxels of J[p, v]^2, computed on the device with
 * FP64 accumulation; synchronous; cached in the handle after the first call.
 */
fft_status fft_frob2(fft_geom g, double* out);

/*
 * fft_cg_solve - damped least squares (Sec. II-D, Eq. leastSquare_misfit with
 * Gamma_n = I, Gamma_pr = I): minimise 1/2 |J m - d|^2 + 1/2 lambda |m|^2 by CGLS,
 * n_iter iterations, no early stop. lambda = lambda_rel * |J|_F^2 / V (the mean diagonal of
 * J^T J), so lambda_rel is dimensionless.
 *   d_dev     device float32[M] data.
 *   m_dev     device float32[V]: in = starting model (zeros for m0 = 0), out = solution.
 *   hist_host nullable host double[n_iter + 1]: |J^T r - lambda m|^2 before each iteration
 *             and after the last.
 * Vectors are FP32; inner products, alpha, beta and gamma are FP64 on the device (no host
 * round trip). The iteration loop is captured once per handle into a CUDA graph and
 * replayed. A vanishing gradient (|J^T r - lambda m|^2 = 0) means m already minimises the
 * misfit: the remaining iterations keep it, and that is not a breakdown.
 * Asynchronous on `stream` when hist_host is NULL: the call returns once the solve is
 * enqueued, and fft_cg_status gives its outcome. With hist_host the call synchronises and
 * returns that outcome itself. The first solve on a handle also computes |J|_F^2
 * (synchronously, then cached) and captures the graph.
 */
fft_status fft_cg_solve(fft_geom g, const float* d_dev, double lambda_rel, int32_t n_iter,
                        float* m_dev, double* hist_host, void* stream);

/*
 * fft_cg_status - outcome of the last fft_cg_solve enqueued on g: synchronises `stream` (the
 * solve's stream), then returns FFT_OK, or FFT_ERR_BREAKDOWN if a curvature was <= 0 with a
 * non-zero gradient or a scalar became non-finite (the iterations after a breakdown leave m
 * unchanged). FFT_OK if g has not solved yet. Each solve resets the flag, so the answer is for
 * the most recent solve only.
 */
fft_status fft_cg_status(fft_geom g, void* stream);

/*
 * fft_cg_continue - n_iter more CGLS iterations (Sec. II-D, Eq. leastSquare_misfit, as in
 * fft_cg_solve) from the state the handle holds (left by the last fft_cg_solve,
 * fft_cg_continue or fft_cg_load on it): the same loop as fft_cg_solve's,
 * so a solve of k iterations continued for n gives the same bits as one solve of k + n.
 *   m_dev     device float32[V], out: the model after the iterations (the state itself stays
 *             in the handle; m_dev is not read).
 *   hist_host nullable host double[n_iter + 1]: |J^T r - lambda m|^2 before the first of these
 *             iterations and after each.
 * Asynchronous and synchronising exactly like fft_cg_solve (a breakdown flag carried in the
 * state stays set: its iterations keep m). FFT_ERR_STATE if the handle holds no CG state.
 */
fft_status fft_cg_continue(fft_geom g, int32_t n_iter, float* m_dev, double* hist_host, void* stream);

/*
 * fft_psf_row_groups - host only (no device work, no handle): the grouping of rows the
 * tensor-core path of fft_psf_batch uses (Sec. II-D, Eq. resolution_2 summed group by group):
 * rows are grouped by the set of subsets that hold them, so that the PSF of subset s is the
 * sum of the groups whose set contains s.
 *   n_rows        rows of the geometry (M).
 *   subset_off, n_subsets, subset_rows   as in fft_psf_batch (1 .. 32 subsets).
 *   grp           host uint8[n_rows] out: group of each row, 0xFF for a row in no subset.
 *   gmask         host uint32[32] out: bit s of gmask[g] set if group g's rows are in subset s;
 *                 groups numbered in order of their first row.
 *   n_groups      out: the number of groups (<= 32), or -1 if there are more than 32 (grp and
 *                 gmask then hold no complete grouping; fft_psf_batch then takes the subsets
 *                 one at a time).
 * FFT_ERR_ARG for a row outside [0, n_rows) or listed twice in one subset.
 */
fft_status fft_psf_row_groups(int64_t n_rows, const int32_t* subset_off, int32_t n_subsets,
                              const int32_t* subset_rows, uint8_t* grp, uint32_t* gmask, int32_t* n_groups);

/*
 * Checkpoint and resume of a solve (plumbing around the CGLS of Sec. II-D; the paper has no
 * counterpart). The state is (m, p, r, gamma, lambda, breakdown flag,
 * iterations done), stored in FP32 / FP64 exactly as the loop keeps it, so a state saved,
 * loaded into a handle of the same geometry and continued gives the same bits as the
 * uninterrupted solve.
 *   fft_cg_state_bytes  *bytes = size of a saved state: a 64-byte header, then m (V floats),
 *                       p (V floats) and r (M floats).
 *   fft_cg_save         copies the handle's state into host_buf (host memory, `bytes` >=
 *                       fft_cg_state_bytes); synchronises `stream`. FFT_ERR_STATE if the
 *                       handle holds no state, FFT_ERR_ARG if the buffer is too small.
 *   fft_cg_load         replaces the handle's state by the one in host_buf (allocating the CG
 *                       workspace on first use); synchronises `stream`. FFT_ERR_ARG if the
 *                       buffer is not a state of fft_cg_save, is short, or was saved for
 *                       another number of rows or voxels.
 */
fft_status fft_cg_state_bytes(fft_geom g, int64_t* bytes);
fft_status fft_cg_save(fft_geom g, void* host_buf, int64_t bytes, void* stream);
fft_status fft_cg_load(fft_geom g, const void* host_buf, int64_t bytes, void* stream);

/*
 * fft_psf_batch - Hessian point-spread functions (Sec. II-D, Eq. resolution_2):
 *   out[(s * n_spike + k) * V + v] = sum_{p in S_s} J[p, v] J[p, spike_vox[k]]
 * i.e. H_S e_k with a unit (1 m/s) spike, for every row subset S_s and spike k.
 *   spike_vox     host int64[n_spike] voxel indices (0 <= . < V), n_spike >= 1.
 *   subset_off    host int32[n_subsets + 1] CSR offsets into subset_rows (subset_off[0] = 0,
 *                 non-decreasing), n_subsets >= 1.
 *   subset_rows   host int32[subset_off[n_subsets]] row indices in [0, M) (each subset ascending).
 *   mode          0: FP32 CUDA cores, one PSF at a time: the column D = J_S e_k (one thread per
 *                    row of S), then a J^T that skips the rows where D is zero.
 *                 1: BF16 tensor cores: Y = J^T D for all n_subsets x n_spike columns of
 *                    D = J_S E at once. Rows are grouped by the set of subsets that hold them
 *                    (nested subsets: one group per subset); D is built as sparse rows with one
 *                    entry per (row, spike), and one persistent kernel generates the J tile of
 *                    each 8 x 4 x 4 voxel brick in FP32, rounds it and D to BF16 and issues
 *                    tcgen05.mma (96 rows of one group per chunk, N = the spikes of a launch)
 *                    accumulating each group in FP32 in its own tensor-memory columns; each
 *                    PSF is the sum of its subset's groups. A launch takes as many spikes as fit
 *                    groups x spikes (rounded up to 16) <= 512 accumulator columns and the
 *                    shared memory (144 with 3 groups and three band tables); more run in
 *                    blocks of spikes. With more than 32 groups the subsets are taken one at
 *                    a time. Relative L2 error ~1e-3 (BF16 operands);
 *                    the cut of a band whose Phi does not vanish at dt_max is taken in FP32
 *                    here (the FP32 paths re-decide it in FP64). At most 32 subsets; a subset
 *                    must not list a row twice (FFT_ERR_ARG). FFT_ERR_TIMEOUT if a bounded wait
 *                    on the tensor cores gave up.
 *                 2: FP32 CUDA cores, four columns per J^T: the columns of D taken in
 *                    (spike, subset) order, four at a time through the four-column J^T
 *                    (fft_JT_apply_batch), so that rows shared by a spike's nested subsets
 *                    are evaluated once. Same accuracy as mode 0.
 *   out_dev       device float32[n_subsets * n_spike * V], written entirely.
 * Allocates its scratch (row lists, the columns of D, staging) with cudaMalloc on every call
 * and synchronises with `stream` before returning; see fft_psf_noalloc for a variant that does
 * neither allocation. Mode 1 keeps one buffer in the handle instead, its candidate records
 * (48 bytes per candidate row of a tile; 16 GB for 384 PSFs over 1.57 M rows and 6.29 M
 * voxels): it grows to the largest call's need, counts in fft_geom_info's scratch_bytes and
 * is freed by fft_geom_destroy.
 */
fft_status fft_psf_batch(fft_geom g, const int64_t* spike_vox, int32_t n_spike,
                         const int32_t* subset_off, int32_t n_subsets,
                         const int32_t* subset_rows, int32_t mode, float* out_dev, void* stream);

/*
 * fft_psf_noalloc - one point-spread function H_S e_k (a single spike k, a single row subset
 * S) computed without allocating any device memory. The paper has no counterpart: this entry
 * point is for callers that must not call the device allocator while they run, such as a
 * service that reserves its device memory up front or code inside another framework's memory
 * pool, where a cudaMalloc (which may also synchronise the device) is not allowed.
 *   spike_vox  voxel index of the unit spike, 0 <= spike_vox < V.
 *   rows_dev   DEVICE int32[n_rows]: the rows of S (any order). Indices outside [0, M) are
 *              skipped; the call then returns FFT_ERR_ARG after finishing.
 *   out_dev    device float32[V], written entirely: out[v] = sum_{p in S} J[p, v] J[p, spike_vox].
 * Scratch is a fixed array inside the library: 4,194,304 floats plus 256 bytes (about 16 MB).
 * It is committed on a device when the first geometry is created there (fft_geom_create looks
 * up its device address, which loads the module that holds it) and stays until the process
 * exits; fft_psf_noalloc itself loads and allocates nothing. Geometries with more than
 * 4,194,304 rows are rejected with FFT_ERR_ARG. All calls share the array (each clears what it
 * uses); calls that overlap on the GPU race, so serialise them. The call copies an error
 * counter to host memory and synchronises with `stream` before returning, so it must not be
 * called while `stream` is being captured into a CUDA graph.
 */
fft_status fft_psf_noalloc(fft_geom g, int64_t spike_vox, const int32_t* rows_dev, int32_t n_rows,
                           float* out_dev, void* stream);

/*
 * fft_tc_selftest - diagnostic for the tensor-core (tcgen05) path: computes one 128 x n x k
 * BF16 product with FP32 accumulation in tensor memory on the current device, from
 * integer-valued operands whose product is exact, and returns the largest absolute difference
 * from the exact result in *max_abs_err (0 when operand layout and descriptors are right).
 *   n in {32, 64, 128, 256}; k a multiple of 16 in [16, 256]. Synchronous.
 * Returns FFT_ERR_TIMEOUT if the bounded wait for the tensor cores gave up.
 */
fft_status fft_tc_selftest(int32_t n, int32_t k, double* max_abs_err);

/* Message of the last failing call on this thread ("" if none). */
const char* fft_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FFT_GB300_H */
