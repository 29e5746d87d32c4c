// Damped least squares by CGLS (Sec. II-D, Eq. leastSquare_misfit with Gamma_n = I,
// Gamma_pr = I, alpha J(dc) = 1/2 lambda |dc|^2): the normal equations
// (J^T J + lambda I) m = J^T d are solved iteratively with J and J^T applied on the fly.
//
// Vectors are FP32; every inner product is accumulated in FP64 by a fixed grid of blocks
// followed by a fixed-order final sum, and alpha, beta, gamma live in FP64 device memory,
// so the loop needs no host round trip and is bit-reproducible. The loop is captured once
// into a CUDA graph (per iteration count) on a private stream and replayed on the caller's
// stream; it touches only the handle's own buffers, so the graph is independent of the
// caller's pointers.
//
// The state between iterations is (m, p, r, gamma, lambda) plus the breakdown flag:
// fft_cg_continue runs more iterations from it, and fft_cg_save / fft_cg_load copy it to and
// from a host buffer (a checkpoint), so that a solve stopped after k iterations and resumed
// for n more gives the same bits as k + n iterations in one call.
#include <cuda_runtime.h>
#include <math.h>

#include <cstring>
#include <vector>

#include "fft_common.cuh"

namespace fftgb {

namespace {

constexpr int DOT_BLOCKS = 1024;
constexpr int DOT_THREADS = 256;
enum { S_GAMMA = 0, S_DELTA = 1, S_ALPHA = 2, S_BETA = 3, S_LAMBDA = 4 };

__device__ double block_reduce(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < DOT_THREADS / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

// part[blk] = sum_i a_i^2 over the block's grid-stride share of a; part[DOT_BLOCKS + blk] for b.
__global__ void dot2_partial_kernel(const float* __restrict__ a, int64_t na, const float* __restrict__ b,
                                    int64_t nb, double* __restrict__ part) {
    __shared__ double sh[DOT_THREADS / 32];
    const int64_t stride = (int64_t)DOT_BLOCKS * DOT_THREADS;
    double sa = 0.0, sb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < na; i += stride) {
        double x = a[i];
        sa += x * x;
    }
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < nb; i += stride) {
        double x = b[i];
        sb += x * x;
    }
    sa = block_reduce(sa, sh);
    sb = block_reduce(sb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sa;
        part[DOT_BLOCKS + blockIdx.x] = sb;
    }
}

__device__ double final_sum(const double* part, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += DOT_THREADS) s += part[i];
    return block_reduce(s, sh);
}

// delta = |q|^2 + lambda |p|^2; alpha = gamma / delta, or breakdown. gamma = 0 is a
// vanishing gradient: m already minimises the damped misfit, alpha = 0 keeps it.
__global__ void cg_alpha_kernel(double* __restrict__ scal, const double* __restrict__ part,
                                int32_t* __restrict__ status) {
    __shared__ double sh[DOT_THREADS / 32];
    double qq = final_sum(part, sh);
    double pp = final_sum(part + DOT_BLOCKS, sh);
    if (threadIdx.x == 0) {
        double delta = qq + scal[S_LAMBDA] * pp;
        double gamma = scal[S_GAMMA];
        scal[S_DELTA] = delta;
        if (*status == 0 && gamma == 0.0) {
            scal[S_ALPHA] = 0.0;
        } else if (*status == 0 && delta > 0.0 && isfinite(delta) && isfinite(gamma)) {
            scal[S_ALPHA] = gamma / delta;
        } else {
            scal[S_ALPHA] = 0.0;
            *status = FFT_ERR_BREAKDOWN;
        }
    }
}

// gamma' = |s|^2; beta = gamma' / gamma; gamma = gamma'; hist[it] = gamma'.
__global__ void cg_beta_kernel(double* __restrict__ scal, const double* __restrict__ part,
                               double* __restrict__ hist, int it, int32_t* __restrict__ status, int first) {
    __shared__ double sh[DOT_THREADS / 32];
    double gn = final_sum(part, sh);
    if (threadIdx.x == 0) {
        if (hist) hist[it] = gn;
        if (first) {
            scal[S_GAMMA] = gn;
            scal[S_BETA] = 0.0;
            if (!isfinite(gn)) *status = FFT_ERR_BREAKDOWN;
        } else {
            double g = scal[S_GAMMA];
            bool ok = (*status == 0) && g > 0.0 && isfinite(gn);
            scal[S_BETA] = ok ? gn / g : 0.0;
            if (ok) scal[S_GAMMA] = gn;
            else if (*status == 0 && !isfinite(gn)) *status = FFT_ERR_BREAKDOWN;
        }
    }
}

__global__ void set_lambda_kernel(double* scal, double lam) { scal[S_LAMBDA] = lam; }

// hist[0] = gamma = |J^T r - lambda m|^2 of the state a continued loop starts from.
__global__ void cg_hist0_kernel(const double* __restrict__ scal, double* __restrict__ hist) { hist[0] = scal[S_GAMMA]; }

// r = d - q
__global__ void residual_kernel(const float* __restrict__ d, const float* __restrict__ q, int64_t M,
                                float* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) r[i] = d[i] - q[i];
}

// s -= lambda m, partial sums of s^2.
__global__ void cg_s_kernel(float* __restrict__ s, const float* __restrict__ m, int64_t V,
                            const double* __restrict__ scal, double* __restrict__ part) {
    __shared__ double sh[DOT_THREADS / 32];
    const double lam = scal[S_LAMBDA];
    const int64_t stride = (int64_t)DOT_BLOCKS * DOT_THREADS;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < V; i += stride) {
        float v = (float)((double)s[i] - lam * (double)m[i]);
        s[i] = v;
        acc += (double)v * (double)v;
    }
    acc = block_reduce(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// m += alpha p; r -= alpha q.
__global__ void cg_update_mr_kernel(float* __restrict__ m, const float* __restrict__ p, int64_t V,
                                    float* __restrict__ r, const float* __restrict__ q, int64_t M,
                                    const double* __restrict__ scal) {
    const double al = scal[S_ALPHA];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride)
        m[i] = (float)((double)m[i] + al * (double)p[i]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        r[i] = (float)((double)r[i] - al * (double)q[i]);
}

// p = s + beta p.
__global__ void cg_update_p_kernel(float* __restrict__ p, const float* __restrict__ s, int64_t V,
                                   const double* __restrict__ scal) {
    const double be = scal[S_BETA];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride)
        p[i] = (float)((double)s[i] + be * (double)p[i]);
}

template <typename T>
fft_status cg_alloc(T** p, size_t n) {
    if (*p) return FFT_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("fft_cg_solve: cudaMalloc failed");
        return FFT_ERR_OOM;
    }
    return FFT_OK;
}

fft_status ensure_workspace(fft_geom g, int32_t n_iter) {
    fft_status rc;
    if ((rc = cg_alloc(&g->cg_r, g->M)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_q, g->M)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_d, g->M)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_s, g->V)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_p, g->V)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_m, g->V)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_scal, 8)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_dots, 2 * DOT_BLOCKS)) != FFT_OK) return rc;
    if ((rc = cg_alloc(&g->cg_status, 1)) != FFT_OK) return rc;
    if (g->cg_hist_cap < n_iter + 1) {
        if (g->cg_hist) cudaFree(g->cg_hist);
        g->cg_hist = nullptr;
        if ((rc = cg_alloc(&g->cg_hist, (size_t)n_iter + 1)) != FFT_OK) return rc;
        g->cg_hist_cap = n_iter + 1;
        // captured loops write the old history buffer: capture again
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
    }
    if (!g->cg_stream) {
        cudaStream_t s;
        FFT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        g->cg_stream = s;
    }
    return FFT_OK;
}

// The iteration loop from the handle's state (m, p, r, gamma, lambda); hist[it + 1] receives
// |s|^2 after iteration it.
fft_status enqueue_iterations(fft_geom g, int32_t n_iter, cudaStream_t st) {
    const int64_t M = g->M, V = g->V;
    fft_status rc;
    for (int32_t it = 0; it < n_iter; ++it) {
        // q = J p; delta = |q|^2 + lambda |p|^2; alpha = gamma / delta
        if ((rc = launch_J(g, g->cg_p, g->cg_q, st)) != FFT_OK) return rc;
        dot2_partial_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(g->cg_q, M, g->cg_p, V, g->cg_dots);
        cg_alpha_kernel<<<1, DOT_THREADS, 0, st>>>(g->cg_scal, g->cg_dots, g->cg_status);
        // m += alpha p; r -= alpha q
        cg_update_mr_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(g->cg_m, g->cg_p, V, g->cg_r, g->cg_q, M,
                                                                g->cg_scal);
        // s = J^T r - lambda m; beta = |s|^2 / gamma; p = s + beta p
        if ((rc = launch_JT(g, g->cg_r, g->cg_s, st)) != FFT_OK) return rc;
        cg_s_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(g->cg_s, g->cg_m, V, g->cg_scal, g->cg_dots);
        cg_beta_kernel<<<1, DOT_THREADS, 0, st>>>(g->cg_scal, g->cg_dots, g->cg_hist, it + 1, g->cg_status, 0);
        cg_update_p_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(g->cg_p, g->cg_s, V, g->cg_scal);
    }
    FFT_CUDA(cudaGetLastError());
    return FFT_OK;
}

// Enqueue the whole solve on `st` using only handle buffers (cg_d, cg_m in; cg_m out).
fft_status enqueue_solve(fft_geom g, int32_t n_iter, cudaStream_t st) {
    const int64_t M = g->M, V = g->V;
    const unsigned rb = (unsigned)ceil_div(M, 256);
    fft_status rc;
    FFT_CUDA(cudaMemsetAsync(g->cg_status, 0, sizeof(int32_t), st));
    // r = d - J m
    if ((rc = launch_J(g, g->cg_m, g->cg_q, st)) != FFT_OK) return rc;
    residual_kernel<<<rb, 256, 0, st>>>(g->cg_d, g->cg_q, M, g->cg_r);
    // s = J^T r - lambda m; gamma = |s|^2; p = s
    if ((rc = launch_JT(g, g->cg_r, g->cg_s, st)) != FFT_OK) return rc;
    cg_s_kernel<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(g->cg_s, g->cg_m, V, g->cg_scal, g->cg_dots);
    cg_beta_kernel<<<1, DOT_THREADS, 0, st>>>(g->cg_scal, g->cg_dots, g->cg_hist, 0, g->cg_status, 1);
    FFT_CUDA(cudaMemcpyAsync(g->cg_p, g->cg_s, sizeof(float) * V, cudaMemcpyDeviceToDevice, st));
    return enqueue_iterations(g, n_iter, st);
}

// Capture `enqueue` (n_iter iterations) into the graph held in *slot unless it already holds
// that many, then launch it on `st`.
template <typename F>
fft_status run_graph(fft_geom g, void** slot, int32_t* slot_iters, int32_t n_iter, F enqueue, cudaStream_t st) {
    if (!*slot || *slot_iters != n_iter) {
        if (*slot) {
            cudaGraphExecDestroy((cudaGraphExec_t)*slot);
            *slot = nullptr;
            *slot_iters = -1;
        }
        cudaStream_t cs = (cudaStream_t)g->cg_stream;
        cudaGraph_t graph = nullptr;
        FFT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        fft_status crc = enqueue(cs);
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (crc != FFT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return crc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        *slot = exec;
        *slot_iters = n_iter;
    }
    FFT_CUDA(cudaGraphLaunch((cudaGraphExec_t)*slot, st));
    return FFT_OK;
}

// Header of a saved CG state (fft_cg_save), followed by m (V floats), p (V) and r (M).
struct CgStateHeader {
    uint32_t magic;      // CG_STATE_MAGIC
    uint32_t version;    // 1
    int64_t n_rows, n_vox;
    int64_t iterations;  // iterations behind the state
    int32_t status;      // 0 or FFT_ERR_BREAKDOWN
    int32_t reserved0;
    double gamma, lambda;
    double reserved1;
};
static_assert(sizeof(CgStateHeader) == 64, "CG state header: 64 bytes");
constexpr uint32_t CG_STATE_MAGIC = 0x47434646u;   // "FFCG"

int64_t cg_state_bytes(fft_geom g) { return (int64_t)sizeof(CgStateHeader) + (int64_t)sizeof(float) * (2 * g->V + g->M); }

}  // namespace

}  // namespace fftgb

using namespace fftgb;

extern "C" fft_status fft_cg_solve(fft_geom g, const float* d_dev, double lambda_rel, int32_t n_iter,
                                   float* m_dev, double* hist_host, void* stream) {
    FFT_API_RANGE("fft_cg_solve");
    FFT_ARG(g && d_dev && m_dev, "fft_cg_solve: null argument");
    FFT_ARG(n_iter >= 0 && n_iter <= 100000, "fft_cg_solve: n_iter must be in [0, 100000]");
    FFT_ARG(lambda_rel >= 0 && isfinite(lambda_rel), "fft_cg_solve: lambda_rel must be >= 0");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_workspace(g, n_iter)) != FFT_OK) return rc;
    double fro = 0.0;
    if ((rc = fft_frob2(g, &fro)) != FFT_OK) return rc;
    const double lam = lambda_rel * fro / (double)g->V;

    g->cg_done = -1;   // the handle's state is overwritten from here on
    FFT_CUDA(cudaMemcpyAsync(g->cg_d, d_dev, sizeof(float) * g->M, cudaMemcpyDeviceToDevice, st));
    FFT_CUDA(cudaMemcpyAsync(g->cg_m, m_dev, sizeof(float) * g->V, cudaMemcpyDeviceToDevice, st));
    set_lambda_kernel<<<1, 1, 0, st>>>(g->cg_scal, lam);
    FFT_CUDA(cudaGetLastError());

    rc = run_graph(g, &g->cg_graph, &g->cg_graph_iters, n_iter,
                   [&](cudaStream_t cs) { return enqueue_solve(g, n_iter, cs); }, st);
    if (rc != FFT_OK) return rc;
    g->cg_done = n_iter;
    FFT_CUDA(cudaMemcpyAsync(m_dev, g->cg_m, sizeof(float) * g->V, cudaMemcpyDeviceToDevice, st));
    if (!hist_host) return FFT_OK;   // asynchronous: fft_cg_status reports the outcome
    FFT_CUDA(cudaMemcpyAsync(hist_host, g->cg_hist, sizeof(double) * (n_iter + 1), cudaMemcpyDeviceToHost, st));
    return fft_cg_status(g, stream);
}

extern "C" fft_status fft_cg_status(fft_geom g, void* stream) {
    FFT_ARG(g, "fft_cg_status: null handle");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    if (!g->cg_status) return FFT_OK;   // no solve yet
    cudaStream_t st = (cudaStream_t)stream;
    int32_t status = 0;
    FFT_CUDA(cudaMemcpyAsync(&status, g->cg_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaStreamSynchronize(st));
    if (status != 0) {
        set_error("fft_cg_solve: breakdown (non-positive curvature or non-finite scalar)");
        return FFT_ERR_BREAKDOWN;
    }
    return FFT_OK;
}

extern "C" fft_status fft_cg_continue(fft_geom g, int32_t n_iter, float* m_dev, double* hist_host, void* stream) {
    FFT_API_RANGE("fft_cg_continue");
    FFT_ARG(g && m_dev, "fft_cg_continue: null argument");
    FFT_ARG(n_iter >= 0 && n_iter <= 100000, "fft_cg_continue: n_iter must be in [0, 100000]");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    if (g->cg_done < 0) {
        set_error("fft_cg_continue: the handle holds no CG state (run fft_cg_solve or fft_cg_load first)");
        return FFT_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_workspace(g, n_iter)) != FFT_OK) return rc;
    rc = run_graph(g, &g->cg_graph_cont, &g->cg_graph_cont_iters, n_iter,
                   [&](cudaStream_t cs) {
                       cg_hist0_kernel<<<1, 1, 0, cs>>>(g->cg_scal, g->cg_hist);
                       return enqueue_iterations(g, n_iter, cs);
                   },
                   st);
    if (rc != FFT_OK) return rc;
    g->cg_done += n_iter;
    FFT_CUDA(cudaMemcpyAsync(m_dev, g->cg_m, sizeof(float) * g->V, cudaMemcpyDeviceToDevice, st));
    if (!hist_host) return FFT_OK;   // asynchronous: fft_cg_status reports the outcome
    FFT_CUDA(cudaMemcpyAsync(hist_host, g->cg_hist, sizeof(double) * (n_iter + 1), cudaMemcpyDeviceToHost, st));
    return fft_cg_status(g, stream);
}

extern "C" fft_status fft_cg_state_bytes(fft_geom g, int64_t* bytes) {
    FFT_ARG(g && bytes, "fft_cg_state_bytes: null argument");
    *bytes = cg_state_bytes(g);
    return FFT_OK;
}

extern "C" fft_status fft_cg_save(fft_geom g, void* host_buf, int64_t bytes, void* stream) {
    FFT_ARG(g && host_buf, "fft_cg_save: null argument");
    FFT_ARG(bytes >= cg_state_bytes(g), "fft_cg_save: buffer smaller than fft_cg_state_bytes");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    if (g->cg_done < 0) {
        set_error("fft_cg_save: the handle holds no CG state (run fft_cg_solve first)");
        return FFT_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double scal[8];
    int32_t status = 0;
    FFT_CUDA(cudaMemcpyAsync(scal, g->cg_scal, sizeof(scal), cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaMemcpyAsync(&status, g->cg_status, sizeof(status), cudaMemcpyDeviceToHost, st));
    unsigned char* buf = static_cast<unsigned char*>(host_buf);
    float* vec = reinterpret_cast<float*>(buf + sizeof(CgStateHeader));
    FFT_CUDA(cudaMemcpyAsync(vec, g->cg_m, sizeof(float) * g->V, cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaMemcpyAsync(vec + g->V, g->cg_p, sizeof(float) * g->V, cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaMemcpyAsync(vec + 2 * g->V, g->cg_r, sizeof(float) * g->M, cudaMemcpyDeviceToHost, st));
    FFT_CUDA(cudaStreamSynchronize(st));
    CgStateHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = CG_STATE_MAGIC;
    h.version = 1;
    h.n_rows = g->M;
    h.n_vox = g->V;
    h.iterations = g->cg_done;
    h.status = status;
    h.gamma = scal[S_GAMMA];
    h.lambda = scal[S_LAMBDA];
    memcpy(buf, &h, sizeof(h));
    return FFT_OK;
}

extern "C" fft_status fft_cg_load(fft_geom g, const void* host_buf, int64_t bytes, void* stream) {
    FFT_ARG(g && host_buf, "fft_cg_load: null argument");
    FFT_ARG(bytes >= (int64_t)sizeof(CgStateHeader), "fft_cg_load: buffer shorter than a CG state header");
    CgStateHeader h;
    memcpy(&h, host_buf, sizeof(h));
    FFT_ARG(h.magic == CG_STATE_MAGIC && h.version == 1, "fft_cg_load: not a CG state saved by fft_cg_save");
    FFT_ARG(h.n_rows == g->M && h.n_vox == g->V, "fft_cg_load: the state is for another geometry size");
    FFT_ARG(bytes >= cg_state_bytes(g), "fft_cg_load: buffer shorter than the state");
    FFT_ARG(h.iterations >= 0 && (h.status == 0 || h.status == FFT_ERR_BREAKDOWN) && h.lambda >= 0.0,
            "fft_cg_load: corrupt CG state header");
    fft_status rc = check_device(g->dev);
    if (rc != FFT_OK) return rc;
    if ((rc = ensure_workspace(g, 0)) != FFT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double scal[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    scal[S_GAMMA] = h.gamma;
    scal[S_LAMBDA] = h.lambda;
    const int32_t status = h.status;
    const float* vec = reinterpret_cast<const float*>(static_cast<const unsigned char*>(host_buf) + sizeof(CgStateHeader));
    FFT_CUDA(cudaMemcpyAsync(g->cg_scal, scal, sizeof(scal), cudaMemcpyHostToDevice, st));
    FFT_CUDA(cudaMemcpyAsync(g->cg_status, &status, sizeof(status), cudaMemcpyHostToDevice, st));
    FFT_CUDA(cudaMemcpyAsync(g->cg_m, vec, sizeof(float) * g->V, cudaMemcpyHostToDevice, st));
    FFT_CUDA(cudaMemcpyAsync(g->cg_p, vec + g->V, sizeof(float) * g->V, cudaMemcpyHostToDevice, st));
    FFT_CUDA(cudaMemcpyAsync(g->cg_r, vec + 2 * g->V, sizeof(float) * g->M, cudaMemcpyHostToDevice, st));
    FFT_CUDA(cudaStreamSynchronize(st));
    g->cg_done = h.iterations;
    return FFT_OK;
}
