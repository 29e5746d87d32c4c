// Phi table by FP64 quadrature on the device (Sec. II-C, Eq. Kernel_freq).
//
// Phi(dt_k) = int_0^inf w^3 W(w) sin(w dt_k) dw / int_0^inf w^2 W(w) dw, dt_k = k dt_max/(n-1).
// One CTA per sample k: its threads stride over the quadrature nodes, each thread sums its
// nodes in order, then a fixed-shape tree reduction combines the threads, so the result is
// the same on every run.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "fft_common.cuh"

namespace fftgb {

namespace {

constexpr int TB_THREADS = 256;
constexpr int N_QUAD_GAUSS = 40000;   // Simpson intervals (even)

__device__ __forceinline__ double w_gauss(double w, double w0, double s) {
    double a = (w - w0) / s, b = (w + w0) / s;
    return exp(-0.5 * a * a) + exp(-0.5 * b * b);
}

__device__ double block_sum(double v, double* sh) {
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = TB_THREADS / 2; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// moment = 2: denominator (dt ignored); moment = 3: numerator at dt.
__global__ void phi_gauss_kernel(double w0, double s, int n, double dt_max, double* out) {
    __shared__ double sh[TB_THREADS];
    const int k = blockIdx.x;
    const double wmax = w0 + 12.0 * s;
    const double dw = wmax / N_QUAD_GAUSS;
    const double dt = (double)k * dt_max / (double)(n - 1);
    double num = 0.0, den = 0.0;
    for (int q = threadIdx.x; q <= N_QUAD_GAUSS; q += TB_THREADS) {
        double w = q * dw;
        double c = (q == 0 || q == N_QUAD_GAUSS) ? 1.0 : ((q & 1) ? 4.0 : 2.0);
        double ww = c * w * w * w_gauss(w, w0, s);
        den += ww;
        num += ww * w * sin(w * dt);
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) out[k] = (k == 0) ? 0.0 : num / den;
}

__global__ void phi_sampled_kernel(const double* om, const double* W, int n_om, int n,
                                   double dt_max, double* out) {
    __shared__ double sh[TB_THREADS];
    const int k = blockIdx.x;
    const double dt = (double)k * dt_max / (double)(n - 1);
    double num = 0.0, den = 0.0;
    for (int q = threadIdx.x; q + 1 < n_om; q += TB_THREADS) {
        double h = om[q + 1] - om[q];
        double a0 = om[q] * om[q] * W[q], a1 = om[q + 1] * om[q + 1] * W[q + 1];
        den += 0.5 * h * (a0 + a1);
        num += 0.5 * h * (a0 * om[q] * sin(om[q] * dt) + a1 * om[q + 1] * sin(om[q + 1] * dt));
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) out[k] = (k == 0) ? 0.0 : num / den;
}

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_table_build(const fft_spectrum* spec, int32_t n_samples, double dt_max,
                                      double* host_out, fft_table* out) {
    FFT_API_RANGE("fft_table_build");
    FFT_ARG(spec && out, "fft_table_build: null spec or out");
    FFT_ARG(n_samples >= 2 && n_samples <= 65536, "fft_table_build: n_samples must be in [2, 65536]");
    FFT_ARG(dt_max > 0 && isfinite(dt_max), "fft_table_build: dt_max must be > 0");
    *out = nullptr;
    int dev = 0;
    FFT_CUDA(cudaGetDevice(&dev));
    fft_table t = new fft_table_s();
    t->dev = dev;
    t->n = n_samples;
    t->dt_max = dt_max;
    t->d_phi = nullptr;
    cudaError_t e = cudaMalloc(&t->d_phi, sizeof(double) * n_samples);
    if (e != cudaSuccess) {
        delete t;
        set_error("fft_table_build: cudaMalloc failed");
        return FFT_ERR_OOM;
    }
    fft_status st = FFT_OK;
    if (spec->kind == 0) {
        if (!(spec->f_center_hz > 0) || !(spec->f_sigma_hz > 0)) {
            set_error("fft_table_build: Gaussian spectrum needs f_center_hz > 0 and f_sigma_hz > 0");
            st = FFT_ERR_ARG;
        } else {
            double w0 = 2.0 * M_PI * spec->f_center_hz, s = 2.0 * M_PI * spec->f_sigma_hz;
            phi_gauss_kernel<<<n_samples, TB_THREADS>>>(w0, s, n_samples, dt_max, t->d_phi);
            e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "phi_gauss_kernel");
        }
    } else if (spec->kind == 1) {
        if (!spec->omega || !spec->weight || spec->n_omega < 2) {
            set_error("fft_table_build: sampled spectrum needs omega, weight and n_omega >= 2");
            st = FFT_ERR_ARG;
        } else {
            for (int i = 0; i + 1 < spec->n_omega && st == FFT_OK; ++i)
                if (!(spec->omega[i + 1] > spec->omega[i])) {
                    set_error("fft_table_build: omega must be strictly ascending");
                    st = FFT_ERR_ARG;
                }
            double *d_om = nullptr, *d_w = nullptr;
            if (st == FFT_OK) {
                size_t bytes = sizeof(double) * spec->n_omega;
                if (cudaMalloc(&d_om, bytes) != cudaSuccess || cudaMalloc(&d_w, bytes) != cudaSuccess) {
                    set_error("fft_table_build: cudaMalloc failed");
                    st = FFT_ERR_OOM;
                } else {
                    e = cudaMemcpy(d_om, spec->omega, bytes, cudaMemcpyHostToDevice);
                    if (e == cudaSuccess) e = cudaMemcpy(d_w, spec->weight, bytes, cudaMemcpyHostToDevice);
                    if (e == cudaSuccess) {
                        phi_sampled_kernel<<<n_samples, TB_THREADS>>>(d_om, d_w, spec->n_omega, n_samples,
                                                                      dt_max, t->d_phi);
                        e = cudaGetLastError();
                    }
                    if (e == cudaSuccess) e = cudaDeviceSynchronize();
                    if (e != cudaSuccess) st = cuda_fail(e, "phi_sampled_kernel");
                }
            }
            cudaFree(d_om);
            cudaFree(d_w);
        }
    } else {
        set_error("fft_table_build: spectrum kind must be 0 (Gaussian) or 1 (sampled)");
        st = FFT_ERR_ARG;
    }
    if (st == FFT_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "fft_table_build");
    }
    if (st == FFT_OK && host_out) {
        e = cudaMemcpy(host_out, t->d_phi, sizeof(double) * n_samples, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "fft_table_build copy-out");
    }
    if (st != FFT_OK) {
        cudaFree(t->d_phi);
        delete t;
        return st;
    }
    *out = t;
    return FFT_OK;
}

extern "C" void fft_table_destroy(fft_table t) {
    if (!t) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != t->dev) cudaSetDevice(t->dev);
    cudaFree(t->d_phi);
    if (cur != t->dev) cudaSetDevice(cur);
    delete t;
}

// Sine-series form of Phi (Sec. II-C stores Phi through the amplitudes and frequencies of
// the sine terms of Eq. Kernel_freq). Both integrals by the rectangle rule on the nodes w_j = j dw; for the
// even Gaussian W the denominator is int_0^inf w^2 W dw = sqrt(2 pi) s (w0^2 + s^2).
extern "C" fft_status fft_trig_build(const fft_spectrum* spec, double dt_max, int32_t n_terms, double* coef_out,
                                     double* dw_out, int32_t* n_terms_out, fft_table* out) {
    FFT_API_RANGE("fft_trig_build");
    FFT_ARG(spec && out, "fft_trig_build: null spec or out");
    FFT_ARG(dt_max > 0 && isfinite(dt_max), "fft_trig_build: dt_max must be > 0");
    FFT_ARG(spec->kind == 0, "fft_trig_build: the sine series needs a Gaussian spectrum (kind 0)");
    FFT_ARG(spec->f_center_hz > 0 && spec->f_sigma_hz > 0 && isfinite(spec->f_center_hz) &&
                isfinite(spec->f_sigma_hz),
            "fft_trig_build: Gaussian spectrum needs f_center_hz > 0 and f_sigma_hz > 0");
    FFT_ARG(n_terms >= 0 && n_terms <= TRIG_MAX_TERMS, "fft_trig_build: n_terms must be in [0, 256]");
    *out = nullptr;
    const double w0 = 2.0 * M_PI * spec->f_center_hz, s = 2.0 * M_PI * spec->f_sigma_hz;
    const double T = fmax(2.0 * dt_max, dt_max + 6.5 / s);   // series period
    const double dw = 2.0 * M_PI / T;
    int n = n_terms;
    if (n == 0) {
        const double nn = ceil((w0 + 5.5 * s) / dw);   // W < 3e-7 beyond
        if (!(nn >= 1.0) || nn > TRIG_MAX_TERMS) {
            set_error("fft_trig_build: the automatic term count exceeds 256 (spectrum too wide for dt_max)");
            return FFT_ERR_ARG;
        }
        n = (int)nn;
    }
    int dev = 0;
    FFT_CUDA(cudaGetDevice(&dev));
    const double den = sqrt(2.0 * M_PI) * s * (w0 * w0 + s * s);
    fft_table t = new fft_table_s();
    t->dev = dev;
    t->n = n;
    t->dt_max = dt_max;
    t->d_phi = nullptr;
    t->kind = PHI_TRIG;
    t->dw = dw;
    t->coef.resize(n);
    for (int j = 1; j <= n; ++j) {
        const double w = j * dw, a = (w - w0) / s, b = (w + w0) / s;
        const double W = exp(-0.5 * a * a) + exp(-0.5 * b * b);
        t->coef[j - 1] = dw * w * w * w * W / den;
    }
    if (coef_out)
        for (int j = 0; j < n; ++j) coef_out[j] = t->coef[j];
    if (dw_out) *dw_out = dw;
    if (n_terms_out) *n_terms_out = n;
    *out = t;
    return FFT_OK;
}
