// Low-rank posterior covariance and resolution (Sec. II-D, Eqs. low_rank, posterior_app,
// resolution_app) with Gamma_pr = I and Gamma_n^{-1} = I / sigma^2, so that the
// prior-preconditioned misfit Hessian is H = J^T J / sigma^2.
//
// Dominant eigenpairs by randomized subspace iteration (Halko, Martinsson and Tropp, SIAM
// Review 53, 2011, Algorithms 4.4 and 5.3):
//   Y = H Omega;  n_power times { Q = orth(Y); Y = H Q };  Q = orth(Y);
//   T = Q^T (H Q) = U diag(l) U^T;  V_k = Q U_k (largest k).
// H is applied four columns at a time with the batch J and J^T kernels. orth is SVQB (Stathopoulos and
// Wu, SIAM J. Sci. Comput. 23, 2002) applied three times: with the Gram matrix G = Y^T Y
// (accumulated in FP64) and its eigendecomposition G = U D U^T, Q = Y U D^{-1/2}, where
// directions with D below 1e-12 max D (numerically in the null space: a block wider than the
// rank of H) are dropped as zero columns, which then give zero Ritz values. The small dense
// steps (the cyclic Jacobi eigensolver) run on the host in FP64 on ell x ell matrices.
//
// Blocks are column-major: column j of a V x n block starts at j * V.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "fft_common.cuh"

namespace fftgb {

namespace {

constexpr int MAX_ELL = 256;
constexpr int GT = 32;            // Gram tile (GT x GT outputs per block)
constexpr int G_ROWS = 64;        // rows staged per step
constexpr int G_CHUNK = 16384;    // rows per block (FP64 partial per block)
constexpr int MM_COLS = 32;       // output columns per thread in the block product

// Partial Gram tiles: part[c][i][j] = sum_{v in chunk c} A[i][v] B[j][v]. F64: products and sums
// in FP64 (for raw H Omega blocks, whose squared entries can fall below the FP32 range);
// else FP32 products summed over G_ROWS rows, then added into FP64 per thread.
template <bool F64>
__global__ void __launch_bounds__(256) gram_kernel(const float* __restrict__ A, int na, const float* __restrict__ B,
                                                   int nb, int64_t V, double* __restrict__ part) {
    __shared__ float sA[G_ROWS][GT + 1];
    __shared__ float sB[G_ROWS][GT + 1];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.z * GT;
    const int64_t r_begin = (int64_t)blockIdx.x * G_CHUNK;
    const int64_t r_end = min(V, r_begin + G_CHUNK);
    // thread (ti, tj) owns outputs (ti + 8 a, tj) for a = 0..3: 8 x 32 threads
    const int tj = tid & 31, ti = tid >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t r0 = r_begin; r0 < r_end; r0 += G_ROWS) {
        for (int e = tid; e < G_ROWS * GT; e += 256) {
            const int rr = e % G_ROWS, cc = e / G_ROWS;
            const int64_t r = r0 + rr;
            sA[rr][cc] = (r < r_end && i0 + cc < na) ? A[(int64_t)(i0 + cc) * V + r] : 0.0f;
            sB[rr][cc] = (r < r_end && j0 + cc < nb) ? B[(int64_t)(j0 + cc) * V + r] : 0.0f;
        }
        __syncthreads();
        if (F64) {
            for (int rr = 0; rr < G_ROWS; ++rr) {
                const double b = (double)sB[rr][tj];
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[a] = fma((double)sA[rr][ti + 8 * a], b, acc[a]);
            }
        } else {
            float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
            for (int rr = 0; rr < G_ROWS; ++rr) {
                const float b = sB[rr][tj];
#pragma unroll
                for (int a = 0; a < 4; ++a) s[a] = fmaf(sA[rr][ti + 8 * a], b, s[a]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] += (double)s[a];
        }
        __syncthreads();
    }
    const int64_t base = (int64_t)blockIdx.x * na * nb;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ti + 8 * a, j = j0 + tj;
        if (i < na && j < nb) part[base + (int64_t)i * nb + j] = acc[a];
    }
}

// out[:, c] = sum_i X[:, i] W[i][c]  (X: V x n_in, W: n_in x n_out row-major FP32, out: V x n_out)
__global__ void __launch_bounds__(256) block_product_kernel(const float* __restrict__ X, int n_in,
                                                            const float* __restrict__ W, int n_out, int64_t V,
                                                            float* __restrict__ out) {
    extern __shared__ float sW[];   // [n_in][MM_COLS]
    const int c0 = blockIdx.y * MM_COLS;
    const int nc = min(MM_COLS, n_out - c0);
    for (int e = threadIdx.x; e < n_in * MM_COLS; e += blockDim.x) {
        const int i = e / MM_COLS, c = e % MM_COLS;
        sW[e] = c < nc ? W[(int64_t)i * n_out + c0 + c] : 0.0f;
    }
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    float acc[MM_COLS];
#pragma unroll
    for (int c = 0; c < MM_COLS; ++c) acc[c] = 0.0f;
    for (int i = 0; i < n_in; ++i) {
        const float x = X[(int64_t)i * V + v];
        const float* w = sW + i * MM_COLS;
#pragma unroll
        for (int c = 0; c < MM_COLS; ++c) acc[c] = fmaf(x, w[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < MM_COLS; ++c)
        if (c < nc) out[(int64_t)(c0 + c) * V + v] = acc[c];
}

// res_v = sum_i d_i V[v, i]^2; post_v = (1 - res_v) / alpha
__global__ void lowrank_diag_kernel(const float* __restrict__ vecs, const double* __restrict__ d, int k, int64_t V,
                                    double alpha, float* __restrict__ post, float* __restrict__ res) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) {
        const double x = (double)vecs[(int64_t)i * V + v];
        s += d[i] * x * x;
    }
    if (res) res[v] = (float)s;
    if (post) post[v] = (float)((1.0 - s) / alpha);
}

// ---- host FP64 dense helpers (n <= MAX_ELL)

// Cyclic Jacobi eigensolver for a symmetric matrix (row-major, destroyed): eigenvalues in w,
// eigenvectors in the columns of U (row-major n x n).
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& U) {
    U.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                (i == j ? diag : off) += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {   // U <- U J
                    const double ukp = U[(size_t)k * n + p], ukq = U[(size_t)k * n + q];
                    U[(size_t)k * n + p] = c * ukp - s * ukq;
                    U[(size_t)k * n + q] = s * ukp + c * ukq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

struct LowrankWork {
    cudaStream_t st;
    int64_t V;
    double* part = nullptr;   // [chunks * MAX_ELL * MAX_ELL]
    int chunks = 0;
    float* wmat = nullptr;    // [MAX_ELL * MAX_ELL]
};

// G = A^T B (na x nb, row-major, FP64) on the device, partials summed on the host in order.
fft_status gram(LowrankWork& W, const float* A, int na, const float* B, int nb, std::vector<double>& G,
                bool f64 = false) {
    dim3 grid((unsigned)W.chunks, (unsigned)ceil_div(na, GT), (unsigned)ceil_div(nb, GT));
    if (f64)
        gram_kernel<true><<<grid, 256, 0, W.st>>>(A, na, B, nb, W.V, W.part);
    else
        gram_kernel<false><<<grid, 256, 0, W.st>>>(A, na, B, nb, W.V, W.part);
    FFT_CUDA(cudaGetLastError());
    std::vector<double> h((size_t)W.chunks * na * nb);
    FFT_CUDA(cudaMemcpyAsync(h.data(), W.part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, W.st));
    FFT_CUDA(cudaStreamSynchronize(W.st));
    G.assign((size_t)na * nb, 0.0);
    for (int c = 0; c < W.chunks; ++c)
        for (size_t e = 0; e < G.size(); ++e) G[e] += h[(size_t)c * na * nb + e];
    return FFT_OK;
}

// out = X Wm (X: V x n_in, Wm: n_in x n_out row-major FP64 -> FP32)
fft_status product(LowrankWork& W, const float* X, int n_in, const std::vector<double>& Wm, int n_out, float* out) {
    std::vector<float> wf(Wm.size());
    for (size_t e = 0; e < wf.size(); ++e) wf[e] = (float)Wm[e];
    FFT_CUDA(cudaMemcpyAsync(W.wmat, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice, W.st));
    const size_t smem = sizeof(float) * (size_t)n_in * MM_COLS;
    dim3 grid((unsigned)ceil_div(W.V, 256), (unsigned)ceil_div(n_out, MM_COLS));
    block_product_kernel<<<grid, 256, smem, W.st>>>(X, n_in, W.wmat, n_out, W.V, out);
    FFT_CUDA(cudaGetLastError());
    FFT_CUDA(cudaStreamSynchronize(W.st));   // wf is reused by the next call
    return FFT_OK;
}

// Q = orth(Y): three SVQB passes, Y -> Q -> Y -> Q (Y is overwritten).
fft_status orthonormalise(LowrankWork& W, float* Y, int n, float* Q) {
    std::vector<double> G, d, U, Wm((size_t)n * n);
    for (int pass = 0; pass < 3; ++pass) {
        float* src = pass == 1 ? Q : Y;
        float* dst = pass == 1 ? Y : Q;
        fft_status rc = gram(W, src, n, src, n, G, pass == 0);
        if (rc != FFT_OK) return rc;
        jacobi_eigen(G, n, d, U);
        double dmax = 0.0;
        for (int i = 0; i < n; ++i) dmax = fmax(dmax, d[i]);
        if (!(dmax > 0.0) || !isfinite(dmax)) {
            set_error("fft_hessian_lowrank: the block to orthonormalise is zero or not finite");
            return FFT_ERR_BREAKDOWN;
        }
        for (int c = 0; c < n; ++c) {
            const double sc = d[c] > 1e-12 * dmax ? 1.0 / sqrt(d[c]) : 0.0;
            for (int i = 0; i < n; ++i) Wm[(size_t)i * n + c] = U[(size_t)i * n + c] * sc;
        }
        if ((rc = product(W, src, n, Wm, n, dst)) != FFT_OK) return rc;
    }
    return FFT_OK;
}

// Y = J^T (J X) for the n columns of X (unscaled by sigma), four columns per application of
// the batch kernels; tmpM holds four columns of length M.
fft_status apply_H(fft_geom g, const float* X, int n, float* Y, float* tmpM, cudaStream_t st) {
    for (int j = 0; j < n; j += 4) {
        const int c = std::min(4, n - j);
        fft_status rc = launch_J_batch(g, X + (int64_t)j * g->V, c, tmpM, st);
        if (rc != FFT_OK) return rc;
        if ((rc = launch_JT_batch(g, tmpM, c, Y + (int64_t)j * g->V, st)) != FFT_OK) return rc;
    }
    return FFT_OK;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_hessian_lowrank(fft_geom g, const float* omega_dev, int32_t ell, int32_t k,
                                          int32_t n_power, double sigma, float* vecs_dev, double* eigvals,
                                          void* stream) {
    FFT_API_RANGE("fft_hessian_lowrank");
    FFT_ARG(g && omega_dev && vecs_dev && eigvals, "fft_hessian_lowrank: null argument");
    FFT_ARG(ell >= 1 && ell <= MAX_ELL && k >= 1 && k <= ell, "fft_hessian_lowrank: need 1 <= k <= ell <= 256");
    FFT_ARG(n_power >= 0 && n_power <= 64, "fft_hessian_lowrank: n_power must be in [0, 64]");
    FFT_ARG(sigma > 0 && isfinite(sigma), "fft_hessian_lowrank: sigma must be > 0");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    LowrankWork W;
    W.st = (cudaStream_t)stream;
    W.V = g->V;
    W.chunks = (int)ceil_div(g->V, G_CHUNK);
    float *Y = nullptr, *Q = nullptr, *tmpM = nullptr;
    const size_t blk = sizeof(float) * (size_t)g->V * ell;
    cudaError_t e = cudaMalloc(&Y, blk);
    if (e == cudaSuccess) e = cudaMalloc(&Q, blk);
    if (e == cudaSuccess) e = cudaMalloc(&tmpM, sizeof(float) * (size_t)g->M * 4);
    if (e == cudaSuccess) e = cudaMalloc(&W.part, sizeof(double) * (size_t)W.chunks * MAX_ELL * MAX_ELL);
    if (e == cudaSuccess) e = cudaMalloc(&W.wmat, sizeof(float) * MAX_ELL * MAX_ELL);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = FFT_ERR_OOM;
        set_error("fft_hessian_lowrank: device allocation failed");
    }
    std::vector<double> T, lam, U;
    if (rc == FFT_OK) rc = apply_H(g, omega_dev, ell, Y, tmpM, W.st);
    for (int it = 0; it < n_power && rc == FFT_OK; ++it) {
        rc = orthonormalise(W, Y, ell, Q);
        if (rc == FFT_OK) rc = apply_H(g, Q, ell, Y, tmpM, W.st);
    }
    if (rc == FFT_OK) rc = orthonormalise(W, Y, ell, Q);
    if (rc == FFT_OK) rc = apply_H(g, Q, ell, Y, tmpM, W.st);    // Y = H Q
    if (rc == FFT_OK) rc = gram(W, Q, ell, Y, ell, T);            // T = Q^T H Q
    if (rc == FFT_OK) {
        for (int i = 0; i < ell; ++i)
            for (int j = i + 1; j < ell; ++j) {
                const double s = 0.5 * (T[(size_t)i * ell + j] + T[(size_t)j * ell + i]);
                T[(size_t)i * ell + j] = T[(size_t)j * ell + i] = s;
            }
        jacobi_eigen(T, ell, lam, U);
        std::vector<int> order(ell);
        for (int i = 0; i < ell; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
        std::vector<double> Uk((size_t)ell * k);
        for (int c = 0; c < k; ++c) {
            eigvals[c] = lam[order[c]] / (sigma * sigma);
            for (int i = 0; i < ell; ++i) Uk[(size_t)i * k + c] = U[(size_t)i * ell + order[c]];
        }
        rc = product(W, Q, ell, Uk, k, vecs_dev);
    }
    if (rc == FFT_OK) {
        e = cudaStreamSynchronize(W.st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fft_hessian_lowrank");
    }
    cudaFree(Y);
    cudaFree(Q);
    cudaFree(tmpM);
    cudaFree(W.part);
    cudaFree(W.wmat);
    return rc;
}

extern "C" fft_status fft_lowrank_diag(fft_geom g, const float* vecs_dev, const double* eigvals, int32_t k,
                                       double alpha, float* post_dev, float* res_dev, void* stream) {
    FFT_API_RANGE("fft_lowrank_diag");
    FFT_ARG(g && vecs_dev && eigvals, "fft_lowrank_diag: null argument");
    FFT_ARG(k >= 1 && k <= MAX_ELL, "fft_lowrank_diag: need 1 <= k <= 256");
    FFT_ARG(alpha > 0 && isfinite(alpha), "fft_lowrank_diag: alpha must be > 0");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    std::vector<double> d(k);
    for (int i = 0; i < k; ++i) d[i] = eigvals[i] / (eigvals[i] + alpha);
    double* dd = nullptr;
    FFT_CUDA(cudaMalloc(&dd, sizeof(double) * k));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dd, d.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        lowrank_diag_kernel<<<(unsigned)ceil_div(g->V, 256), 256, 0, st>>>(vecs_dev, dd, k, g->V, alpha, post_dev,
                                                                         res_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dd);
    if (e != cudaSuccess) return cuda_fail(e, "fft_lowrank_diag");
    return FFT_OK;
}
