// precond.cu -- learned right-diagonal preconditioner m = D y: per-column
// features of G, and the forward, backward and Adam kernels of the small MLP
// (8 -> 64 -> 64 -> 1, tanh hidden layers, softplus output) that maps the
// features to D.  Training and inference both run in these kernels.
//
// Parameter vector (FP32, PDST_MLP_NPARAM entries):
//   mu[8], sigma[8]            feature standardisation (not trained)
//   W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3   (trained, 4,801)
// Model: xh = (f - mu) / sigma; h1 = tanh(W1 xh + b1); h2 = tanh(W2 h1 + b2);
//        z = w3 . h2 + b3; D = softplus(z).  Loss per column: (log D - t)^2.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace pdst {
namespace {

constexpr int NF = PDST_MLP_NFEAT;   // 8
constexpr int NH = PDST_MLP_HIDDEN;  // 64
constexpr int OFF_MU = 0, OFF_SD = NF, OFF_W1 = 2 * NF, OFF_B1 = OFF_W1 + NH * NF,
              OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1, NTRAIN = NPARAM - 2 * NF;
static_assert(NPARAM == PDST_MLP_NPARAM, "parameter layout");

constexpr double FEAT_EPS = 1e-8;   // floor inside the logarithms of the features

// ----------------------------------------------------------------- features

// Pass 1, warp per column j = h*nz + k of G (blocked CSC values, FP64 widening):
// f0 = log(||G_:j|| + eps), f1 = log(1 + rows), f2 = (k + 1/2)/nz,
// f3 = sum G_rj^2 log T(r) / sum G_rj^2 (0 for an empty column),
// f7 = log(max_r |G_rj| + eps).
template <class VT>
__global__ void k_feat1(int32_t n, int nz, const int64_t *__restrict__ cell_rptr,
                        const int32_t *__restrict__ cell_cnt, const int32_t *__restrict__ cell_rows,
                        const VT *__restrict__ valB, const int32_t *__restrict__ row_period,
                        const double *__restrict__ logT, float *feat) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const int64_t h = j / nz;
        const int k = (int)(j - h * nz);
        const int64_t c0 = cell_rptr[h];
        const int cnt = cell_cnt[h];
        const VT *v = valB + c0 * nz + k;
        double s2 = 0.0, st = 0.0, mx = 0.0;
        for (int q = lane; q < cnt; q += 32) {
            const double g = (double)widen(v[(int64_t)q * nz]);
            const double g2 = g * g;
            s2 += g2;
            st += g2 * logT[row_period[cell_rows[c0 + q]]];
            mx = fmax(mx, fabs(g));
        }
        s2 = warp_sum(s2);
        st = warp_sum(st);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            float *f = feat + j * NF;
            f[0] = (float)log(sqrt(s2) + FEAT_EPS);
            f[1] = (float)log1p((double)cnt);
            f[2] = (float)((k + 0.5) / nz);
            f[3] = s2 > 0.0 ? (float)(st / s2) : 0.0f;
            f[7] = (float)log(mx + FEAT_EPS);
        }
    }
}

// Pass 2, thread per column: f4..f6 = log of the mean, min and max of
// (||G_:i|| + eps) over the existing 7-point neighbours i of j.
__global__ void k_feat2(int32_t n, int nx, int ny, int nz, float *feat) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(j % nz);
        const int64_t hh = j / nz;
        const int ix = (int)(hh % nx), iy = (int)(hh / nx);
        const int64_t sy = (int64_t)nx * nz;
        int64_t nb[6];
        int c = 0;
        if (k > 0) nb[c++] = j - 1;
        if (k < nz - 1) nb[c++] = j + 1;
        if (ix > 0) nb[c++] = j - nz;
        if (ix < nx - 1) nb[c++] = j + nz;
        if (iy > 0) nb[c++] = j - sy;
        if (iy < ny - 1) nb[c++] = j + sy;
        double sum = 0.0, mn = 0.0, mx = 0.0;
        for (int i = 0; i < c; ++i) {
            // f0 holds log(norm + eps) in FP32; recover the norm term in FP64
            const double t = exp((double)feat[nb[i] * NF + 0]);
            sum += t;
            mn = i == 0 ? t : fmin(mn, t);
            mx = i == 0 ? t : fmax(mx, t);
        }
        float *f = feat + j * NF;
        if (c > 0) {
            f[4] = (float)log(sum / c);
            f[5] = (float)log(mn);
            f[6] = (float)log(mx);
        } else {
            f[4] = f[5] = f[6] = (float)log(FEAT_EPS);
        }
    }
}

// ---------------------------------------------------------------------- MLP

__device__ __forceinline__ float softplus_f(float z) { return z > 20.f ? z : log1pf(expf(z)); }

// log(softplus(z)) and d log(softplus(z)) / dz, stable for large |z|.
__device__ __forceinline__ void log_softplus(float z, float &y, float &dy) {
    if (z < -20.f) {
        y = z;
        dy = 1.f;
    } else {
        const float sp = softplus_f(z);
        y = logf(sp);
        const float sig = 1.f / (1.f + expf(-z));
        dy = sig / sp;
    }
}

// Per-sample forward pass; the parameters live in shared memory.
struct Act {
    float xh[NF], h1[NH], h2[NH], z;
};

__device__ __forceinline__ void mlp_forward_one(const float *__restrict__ P,
                                                const float *__restrict__ f, Act &a) {
#pragma unroll
    for (int i = 0; i < NF; ++i) a.xh[i] = (f[i] - P[OFF_MU + i]) / P[OFF_SD + i];
    for (int i = 0; i < NH; ++i) {
        float t = P[OFF_B1 + i];
#pragma unroll
        for (int k = 0; k < NF; ++k) t += P[OFF_W1 + i * NF + k] * a.xh[k];
        a.h1[i] = tanhf(t);
    }
    for (int i = 0; i < NH; ++i) {
        float t = P[OFF_B2 + i];
        for (int k = 0; k < NH; ++k) t += P[OFF_W2 + i * NH + k] * a.h1[k];
        a.h2[i] = tanhf(t);
    }
    float z = P[OFF_B3];
    for (int k = 0; k < NH; ++k) z += P[OFF_W3 + k] * a.h2[k];
    a.z = z;
}

__global__ void k_mlp_forward(const float *__restrict__ params, const float *__restrict__ feat,
                              int64_t n, double *D, float *logD) {
    __shared__ float P[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        Act a;
        mlp_forward_one(P, feat + j * NF, a);
        float y, dy;
        log_softplus(a.z, y, dy);
        if (D) D[j] = exp((double)y);
        if (logD) logD[j] = y;
    }
}

// Backward, pass 1 (thread per batch sample): forward, loss and the deltas
// of every layer, written to per-sample scratch rows.
// Scratch row layout: xh[8] h1[64] h2[64] d1[64] d2[64] d3 loss (266 floats).
constexpr int SROW = NF + 4 * NH + 2;

__global__ void k_mlp_bwd_samples(const float *__restrict__ params, const float *__restrict__ feat,
                                  const int32_t *__restrict__ idx, const float *__restrict__ target,
                                  int32_t batch, float *scratch) {
    __shared__ float P[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    const int64_t j = idx[s];
    Act a;
    mlp_forward_one(P, feat + j * NF, a);
    float y, dy;
    log_softplus(a.z, y, dy);
    const float err = y - target[j];
    const float d3 = 2.f * err * dy / (float)batch;   // d(mean loss)/dz
    float *row = scratch + (size_t)s * SROW;
    float *d2 = row + NF + 3 * NH;
    float *d1 = row + NF + 2 * NH;
    for (int i = 0; i < NF; ++i) row[i] = a.xh[i];
    for (int i = 0; i < NH; ++i) {
        row[NF + i] = a.h1[i];
        row[NF + NH + i] = a.h2[i];
        d2[i] = P[OFF_W3 + i] * d3 * (1.f - a.h2[i] * a.h2[i]);
    }
    for (int k = 0; k < NH; ++k) {
        float t = 0.f;
        for (int i = 0; i < NH; ++i) t += P[OFF_W2 + i * NH + k] * d2[i];
        d1[k] = t * (1.f - a.h1[k] * a.h1[k]);
    }
    row[NF + 4 * NH] = d3;
    row[NF + 4 * NH + 1] = err * err;
}

// Backward, pass 2 (thread per trained parameter): gradient of the mean loss
// as a fixed-order sum over the batch (deterministic).  grad[NTRAIN] follows
// the parameter layout from W1; grad[NTRAIN] receives the mean loss.
__global__ void k_mlp_bwd_reduce(const float *__restrict__ scratch, int32_t batch, float *grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > NTRAIN) return;
    float acc = 0.f;
    if (t == NTRAIN) {
        for (int s = 0; s < batch; ++s) acc += scratch[(size_t)s * SROW + NF + 4 * NH + 1];
        grad[NTRAIN] = acc / (float)batch;
        return;
    }
    const int p = t + OFF_W1;
    int a_off, b_off;   // gradient = sum_s row[a_off] * row[b_off] (b_off < 0: 1)
    if (p < OFF_B1) {
        const int i = (p - OFF_W1) / NF, k = (p - OFF_W1) % NF;
        a_off = NF + 2 * NH + i;   // d1[i]
        b_off = k;                 // xh[k]
    } else if (p < OFF_W2) {
        a_off = NF + 2 * NH + (p - OFF_B1);
        b_off = -1;
    } else if (p < OFF_B2) {
        const int i = (p - OFF_W2) / NH, k = (p - OFF_W2) % NH;
        a_off = NF + 3 * NH + i;   // d2[i]
        b_off = NF + k;            // h1[k]
    } else if (p < OFF_W3) {
        a_off = NF + 3 * NH + (p - OFF_B2);
        b_off = -1;
    } else if (p < OFF_B3) {
        a_off = NF + 4 * NH;       // d3
        b_off = NF + NH + (p - OFF_W3);   // h2[k]
    } else {
        a_off = NF + 4 * NH;
        b_off = -1;
    }
    for (int s = 0; s < batch; ++s) {
        const float *row = scratch + (size_t)s * SROW;
        acc += row[a_off] * (b_off >= 0 ? row[b_off] : 1.f);
    }
    grad[t] = acc;
}

__global__ void k_adam(float *params, const float *__restrict__ grad, float *m, float *v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NTRAIN) return;
    const float g = grad[t];
    const float mt = b1 * m[t] + (1.f - b1) * g;
    const float vt = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    params[OFF_W1 + t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

std::mutex g_scratch_mutex;
DevBuf *g_mlp_scratch = nullptr;

}  // namespace
}  // namespace pdst

using namespace pdst;

extern "C" pdst_status pdst_precond_features(pdst_handle_t h, const double *log_periods_host,
                                             float *feat_dev, void *stream) {
    PDST_CHECK_ARG(h && log_periods_host && feat_dev, "pdst_precond_features: NULL argument");
    int dtype = h->vals[PDST_F64].present ? PDST_F64 : h->vals[PDST_F32].present ? PDST_F32 : PDST_BF16;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf logT;
    PDST_TRY(logT.alloc(sizeof(double) * h->n_periods));
    PDST_CUDA(cudaMemcpyAsync(logT.p, log_periods_host, sizeof(double) * h->n_periods,
                              cudaMemcpyHostToDevice, s));
    const int grid = num_sms(h->device) * 8;
    if (dtype == PDST_F64)
        k_feat1<double><<<grid, 256, 0, s>>>(h->n, h->nz, h->cell_rptr.as<int64_t>(),
                                            h->cell_cnt.as<int32_t>(), h->cell_rows.as<int32_t>(),
                                            h->vals[0].bcsc.as<double>(), h->row_period.as<int32_t>(),
                                            logT.as<double>(), feat_dev);
    else if (dtype == PDST_F32)
        k_feat1<float><<<grid, 256, 0, s>>>(h->n, h->nz, h->cell_rptr.as<int64_t>(),
                                           h->cell_cnt.as<int32_t>(), h->cell_rows.as<int32_t>(),
                                           h->vals[1].bcsc.as<float>(), h->row_period.as<int32_t>(),
                                           logT.as<double>(), feat_dev);
    else
        k_feat1<__nv_bfloat16><<<grid, 256, 0, s>>>(
            h->n, h->nz, h->cell_rptr.as<int64_t>(), h->cell_cnt.as<int32_t>(),
            h->cell_rows.as<int32_t>(), h->vals[2].bcsc.as<__nv_bfloat16>(),
            h->row_period.as<int32_t>(), logT.as<double>(), feat_dev);
    k_feat2<<<grid, 256, 0, s>>>(h->n, h->grid.nx, h->grid.ny, h->nz, feat_dev);
    PDST_CUDA(cudaGetLastError());
    PDST_CUDA(cudaStreamSynchronize(s));   // logT is released on return
    return PDST_OK;
}

extern "C" pdst_status pdst_mlp_forward(const float *params_dev, const float *feat_dev, int64_t n,
                                        double *D_dev, float *logD_dev, void *stream) {
    PDST_CHECK_ARG(params_dev && feat_dev && n >= 0 && (D_dev || logD_dev),
                   "pdst_mlp_forward: bad argument");
    if (n == 0) return PDST_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t need = (n + 255) / 256;
    const unsigned grid = (unsigned)std::min<int64_t>(need, (int64_t)num_sms(dev) * 8);
    k_mlp_forward<<<grid, 256, 0, (cudaStream_t)stream>>>(params_dev, feat_dev, n, D_dev, logD_dev);
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}

extern "C" pdst_status pdst_mlp_grad(const float *params_dev, const float *feat_dev,
                                     const int32_t *idx_dev, const float *target_dev,
                                     int32_t batch, float *grad_dev, void *stream) {
    PDST_CHECK_ARG(params_dev && feat_dev && idx_dev && target_dev && grad_dev && batch > 0,
                   "pdst_mlp_grad: bad argument");
    PDST_CHECK_ARG(batch <= (1 << 22), "pdst_mlp_grad: batch must be <= 4194304");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_mlp_scratch) g_mlp_scratch = new DevBuf();
    PDST_TRY(g_mlp_scratch->alloc(sizeof(float) * (size_t)SROW * batch));
    k_mlp_bwd_samples<<<(batch + 127) / 128, 128, 0, s>>>(params_dev, feat_dev, idx_dev, target_dev,
                                                         batch, g_mlp_scratch->as<float>());
    k_mlp_bwd_reduce<<<(NTRAIN + 1 + 127) / 128, 128, 0, s>>>(g_mlp_scratch->as<float>(), batch,
                                                             grad_dev);
    PDST_CUDA(cudaGetLastError());
    PDST_CUDA(cudaStreamSynchronize(s));   // the scratch is shared by all callers
    return PDST_OK;
}

extern "C" pdst_status pdst_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev,
                                     float *v_dev, int64_t step, double lr, double beta1,
                                     double beta2, double eps, void *stream) {
    PDST_CHECK_ARG(params_dev && grad_dev && m_dev && v_dev && step >= 1,
                   "pdst_mlp_adam: bad argument");
    const float c1 = (float)(1.0 - std::pow(beta1, (double)step));
    const float c2 = (float)(1.0 - std::pow(beta2, (double)step));
    k_adam<<<(NTRAIN + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        params_dev, grad_dev, m_dev, v_dev, (float)lr, (float)beta1, (float)beta2, (float)eps, c1,
        c2);
    PDST_CUDA(cudaGetLastError());
    return PDST_OK;
}
